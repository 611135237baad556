"""Shared helpers of the GPU tests (collected by no test runner)."""
import numpy as np

import oracle as O


def first_diff(a: bytes, b: bytes):
    n = min(len(a), len(b))
    x = np.frombuffer(a, np.uint8, count=n)
    y = np.frombuffer(b, np.uint8, count=n)
    d = np.flatnonzero(x != y)
    if d.size:
        return int(d[0])
    return None if len(a) == len(b) else n


def describe_diff(gpu: bytes, ref: bytes) -> str:
    off = first_diff(gpu, ref)
    if off is None:
        return "equal"
    msg = f"len gpu={len(gpu)} oracle={len(ref)}, first difference at byte {off}"
    try:
        data0, offs = O.chunk_table(ref)
        if off >= data0:
            blk = int(np.searchsorted(offs, off - data0, side="right") - 1)
            msg += f" (chunk of block {blk}, +{off - data0 - int(offs[blk])})"
        elif off >= O.HEADER_BYTES:
            msg += f" (offset table entry {(off - O.HEADER_BYTES) // 8})"
        else:
            msg += " (header)"
    except Exception as e:  # pragma: no cover
        msg += f" ({e})"
    return msg


def gpu_compress(field_np, block, kind, eps, eps_mode=O.EPS_REL, stage2=True, range_=-1.0,
                 bound_mode=0, zbits=0, group=1):
    import torch
    from paper_1903_07761_gb300 import cz
    f = torch.from_numpy(np.ascontiguousarray(field_np)).cuda()
    out, nb = cz.compress(f, block=block, kind=kind, eps=eps, eps_mode=eps_mode,
                          stage2=stage2, range_=range_, bound_mode=bound_mode, zero_bits=zbits, group=group)
    torch.cuda.synchronize()
    n = int(nb.item())
    return out[:n].cpu().numpy().tobytes()


def gpu_decompress(stream: bytes):
    import torch
    from paper_1903_07761_gb300 import cz
    s = torch.from_numpy(np.frombuffer(stream, np.uint8).copy()).cuda()
    out = cz.decompress(s, nbytes=len(stream))
    torch.cuda.synchronize()
    return out.cpu().numpy()
