"""Randomised differential test: random small configurations (every block
lane, kind, stage 2 on/off, eps from 0 to 1e-2 in both modes, bit zeroing;
noise, bubble and nearly constant fields) go through the GPU path and the
oracle, and must agree byte for byte: stream, decoded field, random-access
tiles and decoded-block cache tiles.  A fixed seed and case count keep it
deterministic."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

LANES = [(np.float32, 8), (np.float32, 16), (np.float32, 32), (np.float32, 64),
         (np.float64, 8), (np.float64, 16), (np.float64, 32)]


def _case(rng):
    from paper_1903_07761_gb300 import inputs
    dt, B = LANES[rng.integers(len(LANES))]
    nb = [int(rng.integers(1, 4 if B < 64 else 2)) for _ in range(3)]
    shape = tuple(B * k for k in nb)
    which = int(rng.integers(3))
    if which == 0:
        f = rng.standard_normal(shape) * rng.uniform(0.1, 100)
    elif which == 1:
        f = inputs.field(inputs.P, shape, np.float64, seed=int(rng.integers(1 << 30)),
                         nbubbles=int(rng.integers(1, 20)))
    else:
        f = np.full(shape, rng.uniform(-5, 5)) + (rng.random(shape) < 0.01) * rng.standard_normal(shape)
    return dict(f=f.astype(dt), B=B, nb=nb, kind=int(rng.integers(3)), stage2=bool(rng.integers(2)),
                eps=float(rng.choice([0.0, 1e-5, 1e-4, 1e-3, 1e-2])),
                mode=int(rng.choice([O.EPS_REL, O.EPS_ABS])), zbits=int(rng.choice([0, 0, 4, 8])))


def test_random_configurations_agree_with_the_oracle():
    import torch
    from paper_1903_07761_gb300 import cz
    rng = np.random.default_rng(20261204)
    for i in range(150):
        c = _case(rng)
        f, B, nb = c["f"], c["B"], c["nb"]
        what = {k: v for k, v in c.items() if k != "f"} | {"shape": f.shape, "dtype": str(f.dtype), "case": i}
        ref = O.compress(f, B, c["kind"], c["eps"], eps_mode=c["mode"], stage2=c["stage2"], zbits=c["zbits"])
        out, n = cz.compress(torch.from_numpy(f).cuda(), block=B, kind=c["kind"], eps=c["eps"],
                             eps_mode=c["mode"], stage2=c["stage2"], zero_bits=c["zbits"])
        assert out[:int(n.item())].cpu().numpy().tobytes() == ref, what
        want_field = O.decompress(ref)
        rec = cz.decompress(out, nbytes=int(n.item())).cpu().numpy()
        assert np.array_equal(rec.view(np.uint8), want_field.view(np.uint8)), what
        want = want_field.reshape(nb[0], B, nb[1], B, nb[2], B).transpose(0, 2, 4, 1, 3, 5).reshape(-1, B, B, B)
        st = torch.from_numpy(np.frombuffer(ref, np.uint8).copy()).cuda()
        ids = rng.integers(0, want.shape[0], int(rng.integers(1, 6))).astype(np.int32)
        tiles = cz.decompress_blocks(st, torch.from_numpy(ids).cuda()).cpu().numpy()
        assert np.array_equal(tiles.view(np.uint8), want[ids].view(np.uint8)), what
        cache = cz.Cache(8, B, f64=f.dtype == np.float64)
        for _ in range(3):
            ids2 = rng.integers(0, want.shape[0], int(rng.integers(1, 8))).astype(np.int32)
            t2, _ = cache.fetch(st, ids2)
            assert np.array_equal(t2.cpu().numpy().view(np.uint8), want[ids2].view(np.uint8)), what
        cache.close()


# aggregate chunks: the group sizes each lane takes (FP32 64^3: none)
GROUPS = {(np.float32, 8): (4, 8, 16), (np.float32, 16): (4, 8, 16), (np.float32, 32): (4, 8),
          (np.float64, 8): (4, 8, 16), (np.float64, 16): (4, 8, 16), (np.float64, 32): (4,)}


def test_random_group_configurations_agree_with_the_oracle():
    """The same generator with aggregate chunks (stage 2 on, a group size
    the lane takes): stream, decoded field, random-access tiles and cache
    tiles."""
    import torch
    from paper_1903_07761_gb300 import cz
    rng = np.random.default_rng(20261205)
    done = 0
    while done < 60:
        c = _case(rng)
        f, B, nb = c["f"], c["B"], c["nb"]
        gs = GROUPS.get((f.dtype.type, B))
        if not gs:
            continue
        g = int(rng.choice(gs))
        what = {k: v for k, v in c.items() if k != "f"} | {"shape": f.shape, "dtype": str(f.dtype), "group": g,
                                                            "case": done}
        ref = O.compress(f, B, c["kind"], c["eps"], eps_mode=c["mode"], zbits=c["zbits"], group=g)
        out, n = cz.compress(torch.from_numpy(f).cuda(), block=B, kind=c["kind"], eps=c["eps"],
                             eps_mode=c["mode"], zero_bits=c["zbits"], group=g)
        assert out[:int(n.item())].cpu().numpy().tobytes() == ref, what
        want_field = O.decompress(ref)
        rec = cz.decompress(out, nbytes=int(n.item())).cpu().numpy()
        assert np.array_equal(rec.view(np.uint8), want_field.view(np.uint8)), what
        want = want_field.reshape(nb[0], B, nb[1], B, nb[2], B).transpose(0, 2, 4, 1, 3, 5).reshape(-1, B, B, B)
        st = torch.from_numpy(np.frombuffer(ref, np.uint8).copy()).cuda()
        ids = rng.integers(0, want.shape[0], int(rng.integers(1, 6))).astype(np.int32)
        tiles = cz.decompress_blocks(st, torch.from_numpy(ids).cuda()).cpu().numpy()
        assert np.array_equal(tiles.view(np.uint8), want[ids].view(np.uint8)), what
        cache = cz.Cache(8, B, f64=f.dtype == np.float64)
        ids2 = rng.integers(0, want.shape[0], int(rng.integers(1, 8))).astype(np.int32)
        t2, _ = cache.fetch(st, ids2)
        assert np.array_equal(t2.cpu().numpy().view(np.uint8), want[ids2].view(np.uint8)), what
        cache.close()
        done += 1
