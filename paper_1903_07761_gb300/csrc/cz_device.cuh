// cz_device.cuh -- device building blocks of the GB300 wavelet codec.
//
// The kernels (cz_pair.cuh) keep a block in registers spread over the
// threads of a CTA; lines along x cross the lanes of a warp (shuffles),
// lines along y cross warps (shared memory), lines along z stay mostly in
// one thread's registers.
// The 1D wavelet steps below are written once per kind and evaluated in all
// three arrangements with the same operation order, using explicitly
// rounded intrinsics (__fadd_rn, __fmul_rn, ...) that the compiler never
// fuses into multiply-adds.  Every formula follows the paper's wavelet
// families (Sec. 2.3 "Wavelet types"):
//   W4   : 4-point Lagrange prediction of odd samples from even samples,
//          one-sided stencils at the ends of the interval;
//   W4li : W4 prediction plus a lifting update of the even samples whose
//          weights give every synthesis wavelet two vanishing moments;
//   W3ai : average interpolation: coarse = pair average, detail = left
//          sample minus the left-half average of the quadratic through
//          three coarse cell averages.
#pragma once

#include <cstdint>
#include <cuda/atomic>

// Two builds of the kernels live in one library: the exact one (default)
// rounds every operation on its own, in the oracle's order, so streams are
// bit-identical to the oracle's; the fast one (translation units compiled
// with CZ_FAST) lets the compiler contract multiply-adds into fused ones
// (one rounding), which changes coefficients by a few ulps.  The fast build
// gets its own namespaces so that the two sets of kernels never mix.
#ifdef CZ_FAST
#define czd czd_fast
#define czp czp_fast
#endif

namespace czd {

constexpr unsigned FULL = 0xffffffffu;
enum { W4 = 0, W4LI = 1, W3AI = 2 };

// ------------------------------------------------------------ arithmetic
#ifdef CZ_FAST
__device__ __forceinline__ float addx(float a, float b) { return a + b; }
__device__ __forceinline__ double addx(double a, double b) { return a + b; }
__device__ __forceinline__ float subx(float a, float b) { return a - b; }
__device__ __forceinline__ double subx(double a, double b) { return a - b; }
__device__ __forceinline__ float mulx(float a, float b) { return a * b; }
__device__ __forceinline__ double mulx(double a, double b) { return a * b; }
#else
__device__ __forceinline__ float addx(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double addx(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float subx(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double subx(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float mulx(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mulx(double a, double b) { return __dmul_rn(a, b); }
#endif
__device__ __forceinline__ float absx(float a) { return fabsf(a); }
__device__ __forceinline__ double absx(double a) { return fabs(a); }

template <typename T>
__device__ __forceinline__ T shfl(T v, int src) { return __shfl_sync(FULL, v, src); }

// ------------------------------------------------------------ W4 rows
// Lagrange weights x16 of the cubic through four coarse nodes j0..j0+3,
// evaluated at the odd sample k + 1/2 (coarse units):
//   k = 0: x=0.5 on 0..3; interior: x=k+1/2 on k-1..k+2;
//   k = m-2: x on the last four nodes; k = m-1: extrapolation past them.
struct W4Row {
  int j0;
  int w[4];
};

__host__ __device__ constexpr W4Row w4_row(int k, int m)
{
  if (k == 0) return W4Row{0, {5, 15, -5, 1}};
  if (k <= m - 3) return W4Row{k - 1, {-1, 9, 9, -1}};
  if (k == m - 2) return W4Row{m - 4, {1, -5, 15, 5}};
  return W4Row{m - 4, {-5, 21, -35, 35}};
}

// ------------------------------------------------------------ W4li update
// Update of coarse node j: s_j += sum_{t < nt} U_{j, k0+t} d_{k0+t}.
// Detail k updates its two nearest coarse nodes (k, k+1), the last detail
// (m-1, past the last node) updates (m-2, m-1).  The weights solve, per
// detail k,   sum_j U_jk M_j^p = (2k+1)^p  for p = 0, 1,  where M_j^p is the
// p-th moment of the predict-only synthesis scaling function of node j
// (1 at fine position 2j plus column j of the W4 rows at odd positions):
// two vanishing moments for every synthesis wavelet.  Solved here in exact
// integer arithmetic (moments scaled by 16) at compile time.
struct LiSrc {
  int k0, nt;
};

__host__ __device__ constexpr LiSrc li_src(int j, int m)
{
  if (j == 0) return LiSrc{0, 1};
  if (j <= m - 3) return LiSrc{j - 1, 2};
  if (j == m - 2) return LiSrc{m - 3, 3};
  return LiSrc{m - 2, 2};
}

struct Frac {
  long long n, d;
};

__host__ __device__ constexpr long long gcd_ll(long long a, long long b)
{
  if (a < 0) a = -a;
  if (b < 0) b = -b;
  while (b != 0) {
    long long t = a % b;
    a = b;
    b = t;
  }
  return a;
}

// weight of detail k on coarse node j (0/1 if j is not one of its targets)
__host__ __device__ constexpr Frac li_frac(int m, int k, int j)
{
  const int a = (k <= m - 2) ? k : m - 2;
  const int b = a + 1;
  if (j != a && j != b) return Frac{0, 1};
  long long m0a = 16, m0b = 16, m1a = 32LL * a, m1b = 32LL * b;
  for (int r = 0; r < m; ++r) {
    const W4Row row = w4_row(r, m);
    for (int q = 0; q < 4; ++q) {
      const int col = row.j0 + q;
      if (col == a) {
        m0a += row.w[q];
        m1a += (long long)row.w[q] * (2 * r + 1);
      }
      if (col == b) {
        m0b += row.w[q];
        m1b += (long long)row.w[q] * (2 * r + 1);
      }
    }
  }
  const long long r0 = 16, r1 = 16LL * (2 * k + 1);
  long long det = m0a * m1b - m0b * m1a;
  long long num = (j == a) ? (r0 * m1b - m0b * r1) : (m0a * r1 - m1a * r0);
  if (det < 0) {
    det = -det;
    num = -num;
  }
  const long long g = gcd_ll(num, det);
  return Frac{num / (g ? g : 1), det / (g ? g : 1)};
}

template <typename T>
__host__ __device__ constexpr T li_weight(int m, int j, int t)
{
  const LiSrc s = li_src(j, m);
  if (t >= s.nt) return T(0);
  const Frac f = li_frac(m, s.k0 + t, j);
  return (T)f.n / (T)f.d;  // one correctly rounded quotient in T
}

// table for runtime lookups: levels with m = 4, 8, 16, 32 coarse values
// (lines of up to 64 points)
template <typename T>
struct LiTable {
  T u[4][32][3];
};

template <typename T>
__host__ __device__ constexpr LiTable<T> make_li_table()
{
  LiTable<T> tb{};
  for (int mi = 0; mi < 4; ++mi) {
    const int m = 4 << mi;
    for (int j = 0; j < m; ++j)
      for (int t = 0; t < 3; ++t) tb.u[mi][j][t] = li_weight<T>(m, j, t);
  }
  return tb;
}

static __constant__ LiTable<float> c_li_f = make_li_table<float>();
static __constant__ LiTable<double> c_li_d = make_li_table<double>();

template <typename T>
__device__ __forceinline__ T li_lookup(int m, int j, int t);
template <>
__device__ __forceinline__ float li_lookup<float>(int m, int j, int t)
{
  return c_li_f.u[m == 4 ? 0 : (m == 8 ? 1 : (m == 16 ? 2 : 3))][j][t];
}
template <>
__device__ __forceinline__ double li_lookup<double>(int m, int j, int t)
{
  return c_li_d.u[m == 4 ? 0 : (m == 8 ? 1 : (m == 16 ? 2 : 3))][j][t];
}

// ------------------------------------------------------------ W3ai rows
// A_k = a_k + q/8 with q over coarse averages a:
//   k = 0    : q = (3 a_0 - 4 a_1) + a_2
//   interior : q =  a_{k-1} - a_{k+1}
//   k = m-1  : q = (-3 a_{m-1} + 4 a_{m-2}) - a_{m-3}
// Uniform form: x0 = bnd ? a_k : a_s1, x1 = bnd ? a_s1 : a_s2,
//   q = w0 x0 + w1 x1 (+ w2 a_s2 if bnd).
struct AiRow {
  int s1, s2;
  int w0, w1, w2;
  bool bnd;
};

__host__ __device__ constexpr AiRow ai_row(int k, int m)
{
  // (interior rows have weights (1, -1): kernels with compile-time rows
  // evaluate them as one subtraction, which rounds the same way)
  if (k == 0) return AiRow{1, 2, 3, -4, 1, true};
  if (k == m - 1) return AiRow{m - 2, m - 3, -3, 4, -1, true};
  return AiRow{k - 1, k + 1, 1, -1, 0, false};
}

// ------------------------------------------------------------ per-point stencil
// Everything a point at level-local index i (line of n = 2m points) needs,
// computed once per level and reused for every line it touches.
template <typename T>
struct Stencil {
  int i;          // local index
  int p[4];       // W4: local indices of the four coarse sources
  T w[4];         // W4: weights (integers)
  int u[3];       // W4li: local indices of the update sources (details)
  T uw[3];        // W4li: update weights
  int nt;         // W4li: number of update terms
  int s1, s2;     // W3ai: local indices (even) of the two average sources
  T aw[3];        // W3ai: weights
  bool bnd;       // W3ai: boundary row (three terms)
};

template <typename T, int KIND>
__device__ __forceinline__ Stencil<T> make_stencil(int i, int m)
{
  Stencil<T> s;
  s.i = i;
  const int k = i >> 1;
  if (KIND == W4 || KIND == W4LI) {
    const W4Row r = w4_row(k, m);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      s.p[q] = 2 * (r.j0 + q);
      s.w[q] = (T)r.w[q];
    }
  }
  if (KIND == W4LI) {
    const LiSrc ls = li_src(k, m);
    s.nt = ls.nt;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      int kk = ls.k0 + t;
      kk = kk < m ? kk : m - 1;  // unused terms keep a valid index
      s.u[t] = 2 * kk + 1;
      s.uw[t] = li_lookup<T>(m, k, t);
    }
  }
  if (KIND == W3AI) {
    const AiRow r = ai_row(k, m);
    s.s1 = 2 * r.s1;
    s.s2 = 2 * r.s2;
    s.aw[0] = (T)r.w0;
    s.aw[1] = (T)r.w1;
    s.aw[2] = (T)r.w2;
    s.bnd = r.bnd;
  }
  return s;
}

// ((w0 c0 + w1 c1) + w2 c2) + w3 c3, times 1/16
template <typename T>
__device__ __forceinline__ T pred4(const T (&w)[4], T c0, T c1, T c2, T c3)
{
  T p = mulx(w[0], c0);
  p = addx(p, mulx(w[1], c1));
  p = addx(p, mulx(w[2], c2));
  p = addx(p, mulx(w[3], c3));
  return mulx(p, (T)0.0625);
}

// Interior W4 rows have weights (-1, 9, 9, -1).  The products by -1 are
// exact negations, and adding a negation is subtracting, so
// ((-c0 + 9 c1) + 9 c2) + (-c3) rounds exactly like ((9 c1 - c0) + 9 c2) - c3.
template <typename T>
__device__ __forceinline__ T pred4i(T c0, T c1, T c2, T c3)
{
  T p = subx(mulx((T)9, c1), c0);
  p = addx(p, mulx((T)9, c2));
  p = subx(p, c3);
  return mulx(p, (T)0.0625);
}

// a compile-time row: interior rows through pred4i
template <typename T>
__device__ __forceinline__ T pred4r(const W4Row &r, T c0, T c1, T c2, T c3)
{
  if (r.w[0] == -1 && r.w[1] == 9 && r.w[2] == 9 && r.w[3] == -1) return pred4i(c0, c1, c2, c3);
  const T w[4] = {(T)r.w[0], (T)r.w[1], (T)r.w[2], (T)r.w[3]};
  return pred4(w, c0, c1, c2, c3);
}

template <typename T>
__device__ __forceinline__ T li_acc(const Stencil<T> &s, T d0, T d1, T d2)
{
  T acc = mulx(s.uw[0], d0);
  if (s.nt > 1) acc = addx(acc, mulx(s.uw[1], d1));
  if (s.nt > 2) acc = addx(acc, mulx(s.uw[2], d2));
  return acc;
}

// A_k from the pair average a (= a_k) and the two source averages
template <typename T>
__device__ __forceinline__ T ai_pred(const Stencil<T> &s, T a, T a1, T a2)
{
  const T x0 = s.bnd ? a : a1;
  const T x1 = s.bnd ? a1 : a2;
  T q = addx(mulx(s.aw[0], x0), mulx(s.aw[1], x1));
  if (s.bnd) q = addx(q, mulx(s.aw[2], a2));
  return addx(a, mulx(q, (T)0.125));
}

// ============================================================ line steps
// A "getter" g(local_index) returns the current value at that index of the
// line; for warp shuffles every lane must call it the same number of times,
// so the steps below call it unconditionally and select afterwards.

// forward, W4 prediction (also phase 1 of W4li)
template <typename T, class G>
__device__ __forceinline__ T fwd_predict(const Stencil<T> &s, T f, G g)
{
  const T c0 = g(s.p[0]), c1 = g(s.p[1]), c2 = g(s.p[2]), c3 = g(s.p[3]);
  const T d = subx(f, pred4(s.w, c0, c1, c2, c3));
  return (s.i & 1) ? d : f;
}

// forward, W4li update of even points from the predicted details
template <typename T, class G>
__device__ __forceinline__ T fwd_update(const Stencil<T> &s, T f1, G g)
{
  const T d0 = g(s.u[0]), d1 = g(s.u[1]), d2 = g(s.u[2]);
  const T up = addx(f1, li_acc(s, d0, d1, d2));
  return (s.i & 1) ? f1 : up;
}

// inverse, W4li: undo the update on even points
template <typename T, class G>
__device__ __forceinline__ T inv_update(const Stencil<T> &s, T v, G g)
{
  const T d0 = g(s.u[0]), d1 = g(s.u[1]), d2 = g(s.u[2]);
  const T c = subx(v, li_acc(s, d0, d1, d2));
  return (s.i & 1) ? v : c;
}

// inverse, W4 prediction added back to odd points
template <typename T, class G>
__device__ __forceinline__ T inv_predict(const Stencil<T> &s, T v, G g)
{
  const T c0 = g(s.p[0]), c1 = g(s.p[1]), c2 = g(s.p[2]), c3 = g(s.p[3]);
  const T f = addx(v, pred4(s.w, c0, c1, c2, c3));
  return (s.i & 1) ? f : v;
}

// forward W3ai; gp(idx) returns raw samples, ga(idx) returns the pair
// average of the pair starting at even idx (lanes may get it from a
// neighbour that already computed it, shared memory recomputes it).
template <typename T, class GP, class GA>
__device__ __forceinline__ T fwd_ai(const Stencil<T> &s, T f, GP gp, GA ga)
{
  const T pr = gp(s.i ^ 1);
  const bool odd = s.i & 1;
  const T a = mulx(odd ? addx(pr, f) : addx(f, pr), (T)0.5);
  const T a1 = ga(s.s1, a), a2 = ga(s.s2, a);
  const T d = subx(pr, ai_pred(s, a, a1, a2));
  return odd ? d : a;
}

// inverse W3ai: pairs (a_k at even, d_k at odd) -> samples
template <typename T, class G>
__device__ __forceinline__ T inv_ai(const Stencil<T> &s, T v, G g)
{
  const T pr = g(s.i ^ 1);
  const bool odd = s.i & 1;
  const T a = odd ? pr : v;
  const T d = odd ? v : pr;
  const T a1 = g(s.s1), a2 = g(s.s2);
  const T f0 = addx(ai_pred(s, a, a1, a2), d);
  const T f1 = subx(mulx((T)2, a), f0);
  return odd ? f1 : f0;
}

// ============================================================ register lines
// One level of the 1D transform on v[0], v[S], ..., v[(n-1)S] (compile-time
// indices).  Same formulas as above with every branch resolved statically.
template <typename T, int KIND, int B, int S>
__device__ __forceinline__ void fwd_reg(T (&v)[B])
{
  constexpr int n = B / S, m = n / 2;
  if constexpr (KIND == W4 || KIND == W4LI) {
    T d[m];
#pragma unroll
    for (int k = 0; k < m; ++k) {
      const W4Row r = w4_row(k, m);
      d[k] = subx(v[(2 * k + 1) * S],
                  pred4r(r, v[2 * r.j0 * S], v[2 * (r.j0 + 1) * S], v[2 * (r.j0 + 2) * S], v[2 * (r.j0 + 3) * S]));
    }
    if constexpr (KIND == W4LI) {
      T s_[m];
#pragma unroll
      for (int j = 0; j < m; ++j) {
        const LiSrc ls = li_src(j, m);
        T acc = mulx(li_lookup<T>(m, j, 0), d[ls.k0]);
        if (ls.nt > 1) acc = addx(acc, mulx(li_lookup<T>(m, j, 1), d[ls.k0 + 1]));
        if (ls.nt > 2) acc = addx(acc, mulx(li_lookup<T>(m, j, 2), d[ls.k0 + 2]));
        s_[j] = addx(v[2 * j * S], acc);
      }
#pragma unroll
      for (int j = 0; j < m; ++j) v[2 * j * S] = s_[j];
    }
#pragma unroll
    for (int k = 0; k < m; ++k) v[(2 * k + 1) * S] = d[k];
  } else {
    T a[m], d[m];
#pragma unroll
    for (int k = 0; k < m; ++k) a[k] = mulx(addx(v[2 * k * S], v[(2 * k + 1) * S]), (T)0.5);
#pragma unroll
    for (int k = 0; k < m; ++k) {
      const AiRow r = ai_row(k, m);
      T q;
      if (r.bnd) {
        q = addx(mulx((T)r.w0, a[k]), mulx((T)r.w1, a[r.s1]));
        q = addx(q, mulx((T)r.w2, a[r.s2]));
      } else {
        q = subx(a[r.s1], a[r.s2]);  // interior weights (1, -1): both products exact
      }
      d[k] = subx(v[2 * k * S], addx(a[k], mulx(q, (T)0.125)));
    }
#pragma unroll
    for (int k = 0; k < m; ++k) {
      v[2 * k * S] = a[k];
      v[(2 * k + 1) * S] = d[k];
    }
  }
}

template <typename T, int KIND, int B, int S>
__device__ __forceinline__ void inv_reg(T (&v)[B])
{
  constexpr int n = B / S, m = n / 2;
  if constexpr (KIND == W4 || KIND == W4LI) {
    if constexpr (KIND == W4LI) {
      T c[m];
#pragma unroll
      for (int j = 0; j < m; ++j) {
        const LiSrc ls = li_src(j, m);
        T acc = mulx(li_lookup<T>(m, j, 0), v[(2 * ls.k0 + 1) * S]);
        if (ls.nt > 1) acc = addx(acc, mulx(li_lookup<T>(m, j, 1), v[(2 * (ls.k0 + 1) + 1) * S]));
        if (ls.nt > 2) acc = addx(acc, mulx(li_lookup<T>(m, j, 2), v[(2 * (ls.k0 + 2) + 1) * S]));
        c[j] = subx(v[2 * j * S], acc);
      }
#pragma unroll
      for (int j = 0; j < m; ++j) v[2 * j * S] = c[j];
    }
#pragma unroll
    for (int k = 0; k < m; ++k) {
      const W4Row r = w4_row(k, m);
      v[(2 * k + 1) * S] = addx(v[(2 * k + 1) * S], pred4r(r, v[2 * r.j0 * S], v[2 * (r.j0 + 1) * S],
                                                          v[2 * (r.j0 + 2) * S], v[2 * (r.j0 + 3) * S]));
    }
  } else {
    T e[m], o[m];
#pragma unroll
    for (int k = 0; k < m; ++k) {
      const AiRow r = ai_row(k, m);
      const T ak = v[2 * k * S];
      T q;
      if (r.bnd) {
        q = addx(mulx((T)r.w0, ak), mulx((T)r.w1, v[2 * r.s1 * S]));
        q = addx(q, mulx((T)r.w2, v[2 * r.s2 * S]));
      } else {
        q = subx(v[2 * r.s1 * S], v[2 * r.s2 * S]);  // interior weights (1, -1): both products exact
      }
      e[k] = addx(addx(ak, mulx(q, (T)0.125)), v[(2 * k + 1) * S]);
      o[k] = subx(mulx((T)2, ak), e[k]);
    }
#pragma unroll
    for (int k = 0; k < m; ++k) {
      v[2 * k * S] = e[k];
      v[(2 * k + 1) * S] = o[k];
    }
  }
}

// ============================================================ scans
template <typename U>
__device__ __forceinline__ U warp_incl_sum(U v)
{
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const U n = __shfl_up_sync(FULL, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

// Barrier of the NTH threads that use barrier BAR (whole warps): 0 is
// __syncthreads (the whole CTA), others are named barriers of a thread
// group.  The scans below run over the NT threads OFF .. OFF + NT - 1 of
// such a group (OFF a multiple of 32; the defaults: the whole CTA).
template <int BAR, int NTH>
__device__ __forceinline__ void group_sync()
{
  if constexpr (BAR == 0)
    __syncthreads();
  else
    asm volatile("bar.sync %0, %1;" ::"n"(BAR), "n"(NTH) : "memory");
}

// Exclusive prefix of v over the group's threads; tmp >= 33 words.
template <int NT, int BAR = 0, int OFF = 0, typename U>
__device__ __forceinline__ U block_exsum(U v, U *tmp, U &total)
{
  constexpr int NWP = NT / 32;
  const int lane = threadIdx.x & 31, wid = ((int)threadIdx.x - OFF) >> 5;
  const U inc = warp_incl_sum(v);
  if (lane == 31) tmp[wid] = inc;
  group_sync<BAR, NT>();
  if (wid == 0) {
    const U t = lane < NWP ? tmp[lane] : U(0);
    const U ti = warp_incl_sum(t);
    if (lane < NWP) tmp[lane] = ti - t;
    if (lane == NWP - 1) tmp[32] = ti;
  }
  group_sync<BAR, NT>();
  const U r = tmp[wid] + inc - v;
  total = tmp[32];
  group_sync<BAR, NT>();
  return r;
}

// Exclusive prefix with one barrier: every warp adds up the totals of the
// warps before it itself.  tmp (>= NT/32 words) must not be written again
// before the caller's next barrier.
template <int NT, int BAR = 0, int OFF = 0, typename U>
__device__ __forceinline__ U block_exsum_nb(U v, U *tmp, U &total)
{
  constexpr int NWP = NT / 32;
  const int lane = threadIdx.x & 31, wid = ((int)threadIdx.x - OFF) >> 5;
  const U inc = warp_incl_sum(v);
  if (lane == 31) tmp[wid] = inc;
  group_sync<BAR, NT>();
  const U t = lane < NWP ? tmp[lane] : U(0);
  const U ti = warp_incl_sum(t);
  const U before = __shfl_sync(FULL, ti - t, wid);  // exclusive prefix of this warp's total
  total = __shfl_sync(FULL, ti, NWP - 1);
  return before + inc - v;
}

// Both of the scans below with one barrier: the exclusive max of vmax over
// the group's earlier threads (imax if none) and the exclusive min of vmin
// over its later threads (imin if none).  tmp >= 2 * NT/32 words, not
// written again before the caller's next barrier.
template <int NT, int BAR = 0, int OFF = 0>
__device__ __forceinline__ void block_exmax_rexmin_nb(int vmax, int imax, int vmin, int imin, int *tmp, int &exmax,
                                                      int &rexmin)
{
  constexpr int NWP = NT / 32;
  const int lane = threadIdx.x & 31, wid = ((int)threadIdx.x - OFF) >> 5;
  int fwd = vmax, bwd = vmin;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int n = __shfl_up_sync(FULL, fwd, o);
    if (lane >= o) fwd = max(fwd, n);
    const int m = __shfl_down_sync(FULL, bwd, o);
    if (lane + o < 32) bwd = min(bwd, m);
  }
  int ex = __shfl_up_sync(FULL, fwd, 1);
  if (lane == 0) ex = imax;
  int rx = __shfl_down_sync(FULL, bwd, 1);
  if (lane == 31) rx = imin;
  if (lane == 31) tmp[wid] = fwd;       // the warp's max
  if (lane == 0) tmp[NWP + wid] = bwd;  // the warp's min
  group_sync<BAR, NT>();
  int pm = imax, pn = imin;
#pragma unroll
  for (int q = 0; q < NWP; ++q) {
    if (q < wid) pm = max(pm, tmp[q]);
    if (q > wid) pn = min(pn, tmp[NWP + q]);
  }
  exmax = max(pm, ex);
  rexmin = min(pn, rx);
}

// Exclusive max over the group's earlier threads (init if none).
template <int NT, int BAR = 0, int OFF = 0>
__device__ __forceinline__ int block_exmax(int v, int init, int *tmp)
{
  constexpr int NWP = NT / 32;
  const int lane = threadIdx.x & 31, wid = ((int)threadIdx.x - OFF) >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int n = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc = max(inc, n);
  }
  int ex = __shfl_up_sync(FULL, inc, 1);
  if (lane == 0) ex = init;
  if (lane == 31) tmp[wid] = inc;
  group_sync<BAR, NT>();
  if (wid == 0) {
    int t = lane < NWP ? tmp[lane] : init;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int n = __shfl_up_sync(FULL, t, o);
      if (lane >= o) t = max(t, n);
    }
    int e = __shfl_up_sync(FULL, t, 1);
    if (lane == 0) e = init;
    if (lane < NWP) tmp[lane] = e;
  }
  group_sync<BAR, NT>();
  const int r = max(tmp[wid], ex);
  group_sync<BAR, NT>();
  return r;
}

// Exclusive min over the group's later threads (init if none).
template <int NT, int BAR = 0, int OFF = 0>
__device__ __forceinline__ int block_rexmin(int v, int init, int *tmp)
{
  constexpr int NWP = NT / 32;
  const int lane = threadIdx.x & 31, wid = ((int)threadIdx.x - OFF) >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int n = __shfl_down_sync(FULL, inc, o);
    if (lane + o < 32) inc = min(inc, n);
  }
  int ex = __shfl_down_sync(FULL, inc, 1);
  if (lane == 31) ex = init;
  if (lane == 0) tmp[wid] = inc;
  group_sync<BAR, NT>();
  if (wid == 0) {
    int t = lane < NWP ? tmp[lane] : init;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int n = __shfl_down_sync(FULL, t, o);
      if (lane + o < 32) t = min(t, n);
    }
    int e = __shfl_down_sync(FULL, t, 1);
    if (lane == 31 || lane == NWP - 1) e = init;
    if (lane < NWP) tmp[lane] = e;
  }
  group_sync<BAR, NT>();
  const int r = min(tmp[wid], ex);
  group_sync<BAR, NT>();
  return r;
}

// ============================================================ look-back
// Single-pass chained scan with decoupled look-back (Merrill and Garland):
// block b publishes its aggregate, then walks back over predecessors until
// it finds an inclusive prefix.  Flag in the top two bits of a u64.
constexpr unsigned long long LB_AGG = 1ull << 62;
constexpr unsigned long long LB_PRE = 2ull << 62;
constexpr unsigned long long LB_VAL = (1ull << 62) - 1;
constexpr unsigned LB_SPIN_LIMIT = 1u << 22;

// Called by all lanes of one warp; returns the exclusive prefix of `agg`.
// On a wait that exceeds `limit` spins, sets *status (if still 0) to
// `timeout_code` and returns what it has: the caller's output is then
// wrong but the kernel ends.  The spin count and the decision to give up
// are the same in every lane (they follow warp-wide ballots).
// Indices below `first` count as an inclusive prefix of 0 (a segment of
// the state array starts there).
__device__ __forceinline__ unsigned long long lookback(unsigned long long *state, int bid,
                                                       unsigned long long agg,
                                                       unsigned int *status, int timeout_code, int first = 0,
                                                       unsigned limit = LB_SPIN_LIMIT)
{
  const int lane = threadIdx.x & 31;
  using aref = cuda::atomic_ref<unsigned long long, cuda::thread_scope_device>;
  if (lane == 0) aref(state[bid]).store((bid == first ? LB_PRE : LB_AGG) | agg, cuda::memory_order_relaxed);
  unsigned long long excl = 0;
  int base = bid;
  unsigned spins = 0;
  while (base > first) {
    const int j = base - 1 - lane;
    unsigned long long s = LB_PRE;  // before the segment: prefix 0
    if (j >= first) s = aref(state[j]).load(cuda::memory_order_relaxed);
    const unsigned long long flag = s & ~LB_VAL;
    const unsigned pm = __ballot_sync(FULL, flag == LB_PRE);
    const unsigned im = __ballot_sync(FULL, flag == 0);
    const unsigned upto = pm ? (pm & (~pm + 1)) : 0u;  // lowest prefix lane
    const unsigned need = pm ? (upto | (upto - 1)) : FULL;
    if (im & need) {
      if (++spins > limit) {
        if (lane == 0) atomicCAS(status, 0u, (unsigned)timeout_code);
        break;
      }
      __nanosleep(32);
      continue;
    }
    unsigned long long val = ((need >> lane) & 1u) ? (s & LB_VAL) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(FULL, val, o);
    excl += val;
    if (pm) break;
    base -= 32;
  }
  if (lane == 0 && bid != first)
    aref(state[bid]).store(LB_PRE | ((excl + agg) & LB_VAL), cuda::memory_order_relaxed);
  return excl;
}

// min / max that ignore a NaN operand (IEEE minNum / maxNum)
__device__ __forceinline__ float min_nn(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ float max_nn(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double min_nn(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ double max_nn(double a, double b) { return fmax(a, b); }
// three operands (FP32: one instruction; NaN operands are ignored as above)
__device__ __forceinline__ float min3_nn(float a, float b, float c)
{
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ float max3_nn(float a, float b, float c)
{
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ double min3_nn(double a, double b, double c) { return fmin(fmin(a, b), c); }
__device__ __forceinline__ double max3_nn(double a, double b, double c) { return fmax(fmax(a, b), c); }

// ------------------------------------------------------------ order keys
__device__ __forceinline__ unsigned long long order_key(float f)
{
  const unsigned b = __float_as_uint(f);
  return (b & 0x80000000u) ? (unsigned long long)(~b) : (unsigned long long)(b | 0x80000000u);
}
__device__ __forceinline__ unsigned long long order_key(double f)
{
  const unsigned long long b = (unsigned long long)__double_as_longlong(f);
  return (b >> 63) ? ~b : (b | (1ull << 63));
}
__device__ __forceinline__ double key_value(unsigned long long k, float)
{
  const unsigned u = (unsigned)k;
  const unsigned b = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
  return (double)__uint_as_float(b);
}
__device__ __forceinline__ double key_value(unsigned long long k, double)
{
  const unsigned long long b = (k >> 63) ? (k & ~(1ull << 63)) : ~k;
  return __longlong_as_double((long long)b);
}

}  // namespace czd
