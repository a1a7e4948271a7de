// vcycle.cu -- solve-phase V-cycle (Algorithm 1) and the coarsest solvers.
//
// Level k < L, zero initial guess (Algorithm 1 called with x_k = 0, as the
// preconditioner of Algorithms 4-5 and the recursion use it):
//   presmooth  x = omega D^-1 f                      (first damped-Jacobi sweep from 0)
//              x <- x + omega D^-1 (f - A x)         (further sweeps, nu_pre > 1)
//   residual   t = f - A x
//   restrict   f_{k+1}[I] = sum_{i in I} t_i         (members ascending)
//   recurse / coarsest solve  x_{k+1}
//   prolong + postsmooth (fused)  y = xp + omega D^-1 (f - A xp),  xp = x + P x_{k+1}
// Coarsest level: dense inverse times vector, or Jacobi-PCG to 1e-12 (Sec. 4.2).
//
// Every kernel is bandwidth-bound (about 0.16 flop per byte in FP64); rows are
// handled by TPR threads (1 for stencil-like rows), matrix streamed once.
#include <algorithm>
#include <map>
#include <mutex>
#include <functional>
#include <type_traits>
#include <tuple>

#include "common.cuh"

// ---------------------------------------------------------------------------
// Row-kernel helpers
// ---------------------------------------------------------------------------
// Inverse diagonal entry; a null array means a unit diagonal (the scaled
// D^-1/2 A D^-1/2 levels of the FP16-storage mode).
template <typename T>
__device__ __forceinline__ T dval(const T *__restrict__ d, int i) { return d ? __ldg(&d[i]) : T(1); }

__device__ __forceinline__ double as_arith(double v, double) { return v; }
__device__ __forceinline__ float as_arith(float v, float) { return v; }
__device__ __forceinline__ float as_arith(__half v, float) { return __half2float(v); }

// Sum over row entries [b, e) of val * X(col), lanes `sub` of a TPR-wide group.
template <int TPR, typename T, typename V, typename XF>
__device__ __forceinline__ T row_sum(const int32_t *__restrict__ ci, const V *__restrict__ val, int b, int e,
                                     int sub, XF xf) {
  T s = T(0);
  for (int k = b + sub; k < e; k += TPR) s += as_arith(__ldg(&val[k]), T(0)) * xf(__ldg(&ci[k]));
  if (TPR > 1) {
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;
}

// Warp-uniform loop over rows, TPR lanes per row.
#define ROW_LOOP_BEGIN(TPR, n)                                                          \
  const int _lane = threadIdx.x & 31;                                                   \
  const int _sub = _lane & ((TPR)-1);                                                   \
  const long long _rows_per_warp = 32 / (TPR);                                          \
  const long long _nwarps = ((long long)gridDim.x * blockDim.x) >> 5;                   \
  for (long long _base = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * _rows_per_warp; \
       _base < (n); _base += _nwarps * _rows_per_warp) {                                \
    const int _slot = (int)(_base + _lane / (TPR));                                     \
    const bool valid = _slot < (n);                                                     \
    const int row = (valid && perm) ? __ldg(&perm[_slot]) : _slot;
#define ROW_LOOP_END }


// ---------------------------------------------------------------------------
// Row ordering by length class.  A warp issues every FP64 instruction for all
// 32 lanes, so with one thread per row a warp pays for its longest row; on
// irregular (coarse) levels that inflates the FP64 work several times.  Rows
// are therefore processed grouped by length class (class limits grow by 1.5x
// or less), each class in index order: a fixed, deterministic order.
// ---------------------------------------------------------------------------
#define ROW_CLASSES 11
__device__ __forceinline__ int row_class(int len) {
  return len <= 4 ? 0 : len <= 6 ? 1 : len <= 8 ? 2 : len <= 12 ? 3 : len <= 16 ? 4 : len <= 24 ? 5
       : len <= 32 ? 6 : len <= 48 ? 7 : len <= 64 ? 8 : len <= 96 ? 9 : 10;
}

// Exclusive block scan of 0/1 flags; *total receives the block total.
__device__ __forceinline__ int block_scan01(int flag, int *sh, int *total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned m = __ballot_sync(0xffffffffu, flag);
  const int in_warp = __popc(m & ((1u << lane) - 1u));
  if (lane == 0) sh[wid] = __popc(m);
  __syncthreads();
  int off = 0, tot = 0;
  for (int w = 0; w < nw; ++w) {
    const int c = sh[w];
    if (w < wid) off += c;
    tot += c;
  }
  __syncthreads();
  *total = tot;
  return off + in_warp;
}

// ord[0..nr) = local indices 0..nr-1 grouped by length class, stable.
// len_of(k) gives the length of local row k.  All threads of the block call it.
template <typename LenF>
__device__ void block_class_order(int nr, int *ord, int *sh, LenF len_of, int *class_start = nullptr) {
  int base_pos = 0;
  for (int c = 0; c < ROW_CLASSES; ++c) {
    if (class_start && threadIdx.x == 0) class_start[c] = base_pos;
    for (int b0 = 0; b0 < nr; b0 += blockDim.x) {
      const int k = b0 + threadIdx.x;
      const int flag = (k < nr && row_class(len_of(k)) == c) ? 1 : 0;
      int total;
      const int pos = block_scan01(flag, sh, &total);
      if (flag) ord[base_pos + pos] = k;
      base_pos += total;
    }
  }
  if (class_start && threadIdx.x == 0) class_start[ROW_CLASSES] = base_pos;
  __syncthreads();
}

// Setup: perm[w*ORDER_WINDOW + j] = rows of window w grouped by length class.
#define ORDER_WINDOW 4096
__global__ void k_level_order(int n, const int32_t *__restrict__ rp, int32_t *__restrict__ perm) {
  __shared__ int sh[32];
  const int r0 = blockIdx.x * ORDER_WINDOW;
  const int nr = min(ORDER_WINDOW, n - r0);
  if (nr <= 0) return;
  block_class_order(nr, perm + r0, sh, [&](int k) { return rp[r0 + k + 1] - rp[r0 + k]; });
  for (int k = threadIdx.x; k < nr; k += blockDim.x) perm[r0 + k] += r0;
}

// ---------------------------------------------------------------------------
// V-cycle kernels
// ---------------------------------------------------------------------------
// Streaming kernels walk the vectors in rounds of STREAM_U elements per thread
// (i, i + S, i + 2S, ... for S threads in all): every load of a round is in
// flight before the first store, and each load instruction stays coalesced.
#define STREAM_U 4

template <typename T>
__global__ void k_jacobi0(int n, const T *__restrict__ f, const T *__restrict__ dinv, T omega, T *__restrict__ x,
                          const KState *st) {
  if (is_done(st)) return;
  const long long S = (long long)gridDim.x * blockDim.x;
  for (long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; i0 < n; i0 += STREAM_U * S) {
    T fv[STREAM_U], dv[STREAM_U];
#pragma unroll
    for (int u = 0; u < STREAM_U; ++u) {
      const long long i = i0 + u * S;
      if (i < n) {
        fv[u] = f[i];
        dv[u] = dval(dinv, (int)i);
      }
    }
#pragma unroll
    for (int u = 0; u < STREAM_U; ++u) {
      const long long i = i0 + u * S;
      if (i < n) x[i] = omega * (dv[u] * fv[u]);
    }
  }
}

// t = f - A x
template <int TPR, typename T, typename V>
__global__ void k_residual(int n, const int32_t *__restrict__ perm, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           const V *__restrict__ val, const T *__restrict__ x, const T *__restrict__ f,
                           T *__restrict__ t, const KState *st) {
  if (is_done(st)) return;
  ROW_LOOP_BEGIN(TPR, n)
  int b = 0, e = 0;
  if (valid) { b = __ldg(&rp[row]); e = __ldg(&rp[row + 1]); }
  T ax = row_sum<TPR, T, V>(ci, val, b, e, _sub, [&](int j) { return __ldg(&x[j]); });
  if (valid && _sub == 0) t[row] = f[row] - ax;
  ROW_LOOP_END
}

// First presmoothing sweep from the zero guess fused with the residual:
// x = omega D^-1 f (stored) and t = f - A x, neighbours' x formed on the fly.
template <int TPR, typename T, typename V>
__global__ void k_residual0(int n, const int32_t *__restrict__ perm, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            const V *__restrict__ val, const T *__restrict__ dinv, T omega, const T *__restrict__ f,
                            T *__restrict__ x, T *__restrict__ t, const KState *st) {
  if (is_done(st)) return;
  ROW_LOOP_BEGIN(TPR, n)
  int b = 0, e = 0;
  if (valid) { b = __ldg(&rp[row]); e = __ldg(&rp[row + 1]); }
  T ax = row_sum<TPR, T, V>(ci, val, b, e, _sub, [&](int j) { return omega * (dval(dinv, j) * __ldg(&f[j])); });
  if (valid && _sub == 0) {
    const T fi = f[row];
    x[row] = omega * (dval(dinv, row) * fi);
    t[row] = fi - ax;
  }
  ROW_LOOP_END
}

// xout = x + omega D^-1 (f - A x)
template <int TPR, typename T, typename V>
__global__ void k_jacobi(int n, const int32_t *__restrict__ perm, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                         const V *__restrict__ val, const T *__restrict__ dinv, T omega, const T *__restrict__ x,
                         const T *__restrict__ f, T *__restrict__ xout, const KState *st) {
  if (is_done(st)) return;
  ROW_LOOP_BEGIN(TPR, n)
  int b = 0, e = 0;
  if (valid) { b = __ldg(&rp[row]); e = __ldg(&rp[row + 1]); }
  T ax = row_sum<TPR, T, V>(ci, val, b, e, _sub, [&](int j) { return __ldg(&x[j]); });
  if (valid && _sub == 0) xout[row] = x[row] + omega * (dval(dinv, row) * (f[row] - ax));
  ROW_LOOP_END
}

// Residual-operator form of a zero-guess visit (Level documents C and Q).
// t = C f: the residual f - A x of the first damped-Jacobi sweep x = omega
// D^-1 f, in one pass over C (A's pattern) without forming x.
template <int TPR, typename T, typename V>
__global__ void k_op_residual(int n, const int32_t *__restrict__ perm, const int32_t *__restrict__ rp,
                              const int32_t *__restrict__ ci, const V *__restrict__ cval, const T *__restrict__ f,
                              T *__restrict__ t, const KState *st) {
  if (is_done(st)) return;
  ROW_LOOP_BEGIN(TPR, n)
  int b = 0, e = 0;
  if (valid) { b = __ldg(&rp[row]); e = __ldg(&rp[row + 1]); }
  T cf = row_sum<TPR, T, V>(ci, cval, b, e, _sub, [&](int j) { return __ldg(&f[j]); });
  if (valid && _sub == 0) t[row] = cf;
  ROW_LOOP_END
}

// y = Q x_c + wd (f + t): prolongation of the coarse correction and the first
// postsmoothing sweep, x + P x_c + omega D^-1 (f - A (x + P x_c)), in one pass
// over Q (the pattern of A P, n x n_c).
template <int TPR, typename T, typename V>
__global__ void k_op_post(int n, const int32_t *__restrict__ perm, const int32_t *__restrict__ qrp,
                          const int32_t *__restrict__ qci, const V *__restrict__ qval, const T *__restrict__ xc,
                          const T *__restrict__ wd, const T *__restrict__ f, const T *__restrict__ t,
                          T *__restrict__ y, const KState *st) {
  if (is_done(st)) return;
  ROW_LOOP_BEGIN(TPR, n)
  int b = 0, e = 0;
  if (valid) { b = __ldg(&qrp[row]); e = __ldg(&qrp[row + 1]); }
  T qx = row_sum<TPR, T, V>(qci, qval, b, e, _sub, [&](int J) { return __ldg(&xc[J]); });
  if (valid && _sub == 0) y[row] = qx + wd[row] * (f[row] + t[row]);
  ROW_LOOP_END
}

// ---------------------------------------------------------------------------
// TMA-staged row kernels (lanes-per-row choice 0): each block walks tiles of
// ST_ROWS consecutive rows; one elected thread copies a tile's values and
// column indices into shared memory with cp.async.bulk (completion counted
// by an mbarrier), double-buffered so the next tile streams in while the
// current one is computed, and every thread then forms its row's sum from
// shared memory.  This replaces the per-thread, uncoalesced row reads of the
// one-lane kernels.  Waits are bounded: a copy that does not complete within
// about a second sets the timeout flag and the block stops.
// ---------------------------------------------------------------------------
#define ST_ROWS 256
// dynamic shared memory limit of the staged kernels (one value for every level:
// the attribute belongs to the kernel, not to a launch)
#define ST_SMEM_MAX (96 * 1024)
#define ST_WAIT_LIMIT (1ll << 31)

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// bounded wait for a phase of the barrier; false when it gave up
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > ST_WAIT_LIMIT) return false;
  return true;
}

// Byte layout of one stage buffer for a tile of at most `cap` stored entries.
// (the aligned copy of a tile holding `cap` entries spans at most cap + 2*VA - 2
// values and cap + 6 columns)
template <typename V>
__host__ __device__ __forceinline__ size_t st_val_bytes(int cap) {
  return ((size_t)(cap + 2 * (16 / sizeof(V))) * sizeof(V) + 127) / 128 * 128;
}
__host__ __device__ __forceinline__ size_t st_col_bytes(int cap) { return ((size_t)(cap + 8) * 4 + 127) / 128 * 128; }

// largest number of stored entries in a tile of ST_ROWS rows
__global__ void k_tile_max(int n, const int32_t *__restrict__ rp, int *out) {
  const int ntiles = (n + ST_ROWS - 1) / ST_ROWS;
  int m = 0;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x)
    m = max(m, rp[min(n, (t + 1) * ST_ROWS)] - rp[t * ST_ROWS]);
  atomicMax(out, m);
}

// MODE 0: out = f - A x.  MODE 1: out = x + omega D^-1 (f - A x).
template <typename T, typename V, int MODE>
__global__ void __launch_bounds__(ST_ROWS)
    k_rows_staged(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const V *__restrict__ val,
                  const T *__restrict__ dinv, T omega, const T *__restrict__ x, const T *__restrict__ f,
                  T *__restrict__ out, int cap, unsigned *eflags, const KState *st) {
  if (is_done(st)) return;
  extern __shared__ __align__(128) unsigned char st_smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  const size_t vb = st_val_bytes<V>(cap), cb = st_col_bytes(cap);
  V *sval[2] = {(V *)st_smem, (V *)(st_smem + vb + cb)};
  int *scol[2] = {(int *)(st_smem + vb), (int *)(st_smem + 2 * vb + cb)};
  constexpr int VA = 16 / sizeof(V);  // values per 16 bytes
  const int ntiles = (n + ST_ROWS - 1) / ST_ROWS;
  if (threadIdx.x == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // one elected thread issues a tile's copies (16-byte aligned start and size;
  // the arrays are padded, so rounding the end up stays inside them)
  auto issue = [&](int tile, int b) {
    const int r0 = tile * ST_ROWS, r1 = min(n, r0 + ST_ROWS);
    const int e0 = rp[r0], e1 = rp[r1];
    const int v0 = e0 & ~(VA - 1), v1 = (e1 + VA - 1) & ~(VA - 1);
    const int c0 = e0 & ~3, c1 = (e1 + 3) & ~3;
    const unsigned vbytes = (unsigned)(v1 - v0) * sizeof(V), cbytes = (unsigned)(c1 - c0) * 4u;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&mbar[b], vbytes + cbytes);
    if (vbytes) bulk_g2s(sval[b], val + v0, vbytes, &mbar[b]);
    if (cbytes) bulk_g2s(scol[b], ci + c0, cbytes, &mbar[b]);
  };
  unsigned parity[2] = {0u, 0u};
  int k = 0;
  if (threadIdx.x == 0 && (int)blockIdx.x < ntiles) issue(blockIdx.x, 0);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
    const int b = k & 1;
    const int next = tile + gridDim.x;
    if (threadIdx.x == 0 && next < ntiles) issue(next, b ^ 1);
    const bool ok = mbar_wait(&mbar[b], parity[b]);
    parity[b] ^= 1u;
    if (__syncthreads_or(!ok)) {
      // give up: flag it, wait (bounded) for the other buffer's copy, stop
      if (threadIdx.x == 0) {
        atomicOr(eflags, AMG_EFLAG_TIMEOUT);
        if (next < ntiles) mbar_wait(&mbar[b ^ 1], parity[b ^ 1]);
      }
      return;
    }
    const int r0 = tile * ST_ROWS;
    const int row = r0 + threadIdx.x;
    if (row < n) {
      const int e0t = rp[r0];
      const int v0 = e0t & ~(VA - 1), c0 = e0t & ~3;
      const int eb = rp[row], ee = rp[row + 1];
      const V *lv = sval[b] - v0;
      const int *lc = scol[b] - c0;
      T ax = T(0);
      for (int e = eb; e < ee; ++e) ax += as_arith(lv[e], T(0)) * __ldg(&x[lc[e]]);
      if (MODE == 0) out[row] = f[row] - ax;
      else out[row] = x[row] + omega * (dval(dinv, row) * (f[row] - ax));
    }
    __syncthreads();  // buffer b is refilled two tiles later
  }
}

// Scaled levels exist only in the FP16-storage mode, whose vectors are FP32.
// FP64 kernels compile the scaling out: the compiler turns the pointer tests
// into predication, and on this GPU a predicated-off FP64 instruction (here
// the float-to-double conversion and the multiply) still occupies the slow
// FP64 pipe -- it made the FP64 prolongation FP64-bound at a third of the
// HBM rate.
template <typename T>
struct MayScale { static constexpr bool value = !std::is_same<T, double>::value; };

// Coarse correction of fine row i: x_c[agg_i], times isig_c[agg_i] when the
// coarse level is scaled and times sig_i when the fine level is scaled.
template <typename T>
__device__ __forceinline__ T coarse_corr(const T *__restrict__ xc, const int32_t *__restrict__ agg,
                                         const float *__restrict__ sig, const float *__restrict__ isig_c, int i) {
  const int a = __ldg(&agg[i]);
  T c = __ldg(&xc[a]);
  if constexpr (MayScale<T>::value) {
    if (isig_c) c *= (T)__ldg(&isig_c[a]);
    if (sig) c *= (T)__ldg(&sig[i]);
  }
  return c;
}

// Prolongation fused into the first post-smoothing sweep:
// xp = x + P xc; xout = xp + omega D^-1 (f - A xp)
template <int TPR, typename T, typename V>
__global__ void k_prolong_jacobi(int n, const int32_t *__restrict__ perm, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                 const V *__restrict__ val, const T *__restrict__ dinv, T omega,
                                 const T *__restrict__ x, const int32_t *__restrict__ agg,
                                 const T *__restrict__ xc, const float *__restrict__ sig,
                                 const float *__restrict__ isig_c, const T *__restrict__ f, T *__restrict__ xout,
                                 const KState *st) {
  if (is_done(st)) return;
  ROW_LOOP_BEGIN(TPR, n)
  int b = 0, e = 0;
  if (valid) { b = __ldg(&rp[row]); e = __ldg(&rp[row + 1]); }
  T ax = row_sum<TPR, T, V>(ci, val, b, e, _sub,
                            [&](int j) { return __ldg(&x[j]) + coarse_corr(xc, agg, sig, isig_c, j); });
  if (valid && _sub == 0) {
    T xp = x[row] + coarse_corr(xc, agg, sig, isig_c, row);
    xout[row] = xp + omega * (dval(dinv, row) * (f[row] - ax));
  }
  ROW_LOOP_END
}

template <typename T>
__global__ void k_prolong(int n, const T *__restrict__ x, const int32_t *__restrict__ agg, const T *__restrict__ xc,
                          const float *__restrict__ sig, const float *__restrict__ isig_c, T *__restrict__ xout,
                          const KState *st) {
  if (is_done(st)) return;
  const long long S = (long long)gridDim.x * blockDim.x;
  for (long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; i0 < n; i0 += STREAM_U * S) {
    // the round's aggregate ids and x first (read once: streaming loads),
    // then the dependent gathers of x_c, so both waits overlap across the round
    T xv[STREAM_U], cv[STREAM_U];
    int a[STREAM_U];
#pragma unroll
    for (int u = 0; u < STREAM_U; ++u) {
      const long long i = i0 + u * S;
      a[u] = i < n ? __ldcs(&agg[i]) : 0;
    }
#pragma unroll
    for (int u = 0; u < STREAM_U; ++u) {
      const long long i = i0 + u * S;
      xv[u] = i < n ? __ldcs(&x[i]) : T(0);
    }
#pragma unroll
    for (int u = 0; u < STREAM_U; ++u) {
      const long long i = i0 + u * S;
      T c = __ldg(&xc[a[u]]);
      if constexpr (MayScale<T>::value) {
        if (i < n) {
          if (isig_c) c *= (T)__ldg(&isig_c[a[u]]);
          if (sig) c *= (T)__ldg(&sig[i]);
        }
      }
      cv[u] = c;
    }
#pragma unroll
    for (int u = 0; u < STREAM_U; ++u) {
      const long long i = i0 + u * S;
      if (i < n) xout[i] = xv[u] + cv[u];
    }
  }
}

// f_c[I] = sum of t over the members of I, members ascending (each term times
// sig_i on a scaled fine level; the sum times isig_c[I] on a scaled coarse level).
template <typename T>
__global__ void k_restrict(int nc, const int32_t *__restrict__ mrp, const int32_t *__restrict__ mem,
                           const T *__restrict__ t, const float *__restrict__ sig, const float *__restrict__ isig_c,
                           T *__restrict__ fc, const KState *st) {
  if (is_done(st)) return;
  for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += gridDim.x * blockDim.x) {
    int b = mrp[I], e = mrp[I + 1];
    int i = mem[b];
    if constexpr (MayScale<T>::value) {
      T s = sig ? t[i] * (T)sig[i] : t[i];
      for (int k = b + 1; k < e; ++k) {
        i = mem[k];
        s += sig ? t[i] * (T)sig[i] : t[i];
      }
      fc[I] = isig_c ? s * (T)isig_c[I] : s;
    } else {
      T s = t[i];
      for (int k = b + 1; k < e; ++k) s += t[mem[k]];
      fc[I] = s;
    }
  }
}

// b = (B)(a * scale) with an optional per-entry scale
// FP64 <-> FP32 conversions on the integer pipe.  The conversion instructions
// issue on GB300's FP64 pipe (about one per clock per SM), which made the
// precision casts of the V-cycle FP64-bound; these compute the same IEEE
// results from the bit patterns for normal numbers (round to nearest even
// for FP64 -> FP32) and leave zeros, subnormals, infinities and NaNs to the
// instruction.
__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff) - 1023 + 127;  // FP32 biased exponent
  if (e < 1 || e > 254) return (float)x;                 // outside the FP32 normal range
  const unsigned long long mant = b & 0xfffffffffffffull;
  unsigned m = (unsigned)(mant >> 29);
  const unsigned long long rem = mant & 0x1fffffffull, half = 0x10000000ull;
  unsigned r = ((unsigned)e << 23) + m;  // exponent and mantissa, a carry moves into the exponent
  if (rem > half || (rem == half && (m & 1u))) ++r;
  if ((r >> 23) >= 255u) return (float)x;  // rounded up into the infinity range
  return __uint_as_float(r | ((unsigned)(b >> 63) << 31));
}
__device__ __forceinline__ double f32_to_f64(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned e = (b >> 23) & 0xffu;
  if (e == 0u || e == 255u) return (double)x;  // zero, subnormal, infinity, NaN
  const unsigned long long d = ((unsigned long long)(b >> 31) << 63) |
                               ((unsigned long long)(e - 127u + 1023u) << 52) |
                               ((unsigned long long)(b & 0x7fffffu) << 29);
  return __longlong_as_double((long long)d);
}
__device__ __forceinline__ float to_f32(double x) { return f64_to_f32(x); }
__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return f32_to_f64(x); }
__device__ __forceinline__ double to_f64(double x) { return x; }

// b = a (times scale in FP32 when given), converted to B.
template <typename A, typename B>
__global__ void k_cast_scale(int n, const A *__restrict__ a, const float *__restrict__ scale, B *__restrict__ b,
                             const KState *st) {
  if (is_done(st)) return;
  const long long S = (long long)gridDim.x * blockDim.x;
  for (long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; i0 < n; i0 += STREAM_U * S) {
    float av[STREAM_U];
#pragma unroll
    for (int u = 0; u < STREAM_U; ++u) {
      const long long i = i0 + u * S;
      if (i < n) av[u] = scale ? to_f32(a[i]) * scale[i] : to_f32(a[i]);
    }
#pragma unroll
    for (int u = 0; u < STREAM_U; ++u) {
      const long long i = i0 + u * S;
      if (i < n) b[i] = std::is_same<B, double>::value ? (B)to_f64(av[u]) : (B)av[u];
    }
  }
}

// Level 0 of the FP32 cycle in the residual-operator form writes the FP64
// result itself: y is widened as it is written, with the conversion the cast
// kernel uses, which saves a pass over the level-0 vectors.  (Reading the FP64
// right-hand side in the first kernel as well was measured slower on the
// 7-point systems: its neighbour gathers then move twice the bytes.)
template <int TPR>
__global__ void k_op_post_out64(int n, const int32_t *__restrict__ perm, const int32_t *__restrict__ qrp,
                                const int32_t *__restrict__ qci, const float *__restrict__ qval,
                                const float *__restrict__ xc, const float *__restrict__ wd,
                                const float *__restrict__ f, const float *__restrict__ t, double *__restrict__ y,
                                const KState *st) {
  if (is_done(st)) return;
  ROW_LOOP_BEGIN(TPR, n)
  int b = 0, e = 0;
  if (valid) { b = __ldg(&qrp[row]); e = __ldg(&qrp[row + 1]); }
  float qx = row_sum<TPR, float, float>(qci, qval, b, e, _sub, [&](int J) { return __ldg(&xc[J]); });
  if (valid && _sub == 0) y[row] = to_f64(qx + wd[row] * (f[row] + t[row]));
  ROW_LOOP_END
}

// ---------------------------------------------------------------------------
// Coarsest solve: dense inverse (one warp per row, FP64 accumulation)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_gemv_dense(int m, const double *__restrict__ ainv, const T *__restrict__ f, T *__restrict__ x,
                             const KState *st) {
  if (is_done(st)) return;
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  // rows read as double2 when every row starts on 16 bytes (two partial sums
  // per lane), else one element at a time
  const bool vec = (m % 2) == 0 && ((uintptr_t)ainv & 15) == 0;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < m; i += warps) {
    const double *row = ainv + (size_t)i * m;
    double s = 0.0;
    if (vec) {
      const double2 *row2 = (const double2 *)row;
      double s1 = 0.0;
#pragma unroll 4
      for (int q = lane; q < m / 2; q += 32) {
        const double2 a = __ldg(&row2[q]);
        s = __fma_rn(a.x, (double)__ldg(&f[2 * q]), s);
        s1 = __fma_rn(a.y, (double)__ldg(&f[2 * q + 1]), s1);
      }
      s += s1;
    } else {
      for (int j = lane; j < m; j += 32) s += __ldg(&row[j]) * (double)__ldg(&f[j]);
    }
    s = warp_sum(s);
    if (lane == 0) x[i] = (T)s;
  }
}

// Coarsest solve with the FP32 inverse X: xw = (add ? xw : 0) + X v, with FP32
// products and sums (X itself holds only FP32 accuracy), warp per row; the
// last step also writes x = xw in the vector type T.
template <typename V, typename T>
__global__ void k_gemv32(int m, const float *__restrict__ X, const V *__restrict__ v, double *__restrict__ xw,
                         int add, T *__restrict__ xout, const KState *st) {
  if (is_done(st)) return;
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  // rows (and an FP32 v) read as float4 when every row starts on 16 bytes
  // (four partial sums per lane), in batches of GEMV_BATCH loads per lane
  // issued before their products so that enough of the row is in flight;
  // else one element at a time
  constexpr int GEMV_BATCH = 8;
  const bool vec = (m % 4) == 0 && ((uintptr_t)X & 15) == 0 &&
                   (!std::is_same<V, float>::value || ((uintptr_t)v & 15) == 0);
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < m; i += warps) {
    const float *row = X + (size_t)i * m;
    float s = 0.0f;
    if (vec) {
      const float4 *row4 = (const float4 *)row;
      const int m4 = m / 4;
      float s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
      for (int q0 = lane; q0 < m4; q0 += 32 * GEMV_BATCH) {
        float4 a[GEMV_BATCH], b[GEMV_BATCH];
#pragma unroll
        for (int u = 0; u < GEMV_BATCH; ++u) {
          const int q = q0 + 32 * u;
          a[u] = q < m4 ? __ldg(&row4[q]) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < GEMV_BATCH; ++u) {
          const int q = q0 + 32 * u;
          if constexpr (std::is_same<V, float>::value) {
            b[u] = q < m4 ? __ldg(&((const float4 *)v)[q]) : make_float4(0.f, 0.f, 0.f, 0.f);
          } else {
            b[u] = q < m4 ? make_float4((float)v[4 * q], (float)v[4 * q + 1], (float)v[4 * q + 2], (float)v[4 * q + 3])
                          : make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
#pragma unroll
        for (int u = 0; u < GEMV_BATCH; ++u) {
          s = fmaf(a[u].x, b[u].x, s);
          s1 = fmaf(a[u].y, b[u].y, s1);
          s2 = fmaf(a[u].z, b[u].z, s2);
          s3 = fmaf(a[u].w, b[u].w, s3);
        }
      }
      s = (s + s1) + (s2 + s3);
    } else {
      for (int j = lane; j < m; j += 32) s = fmaf(__ldg(&row[j]), (float)v[j], s);
    }
    s = warp_sum(s);
    if (lane == 0) {
      const double xi = (add ? xw[i] : 0.0) + to_f64(s);
      xw[i] = xi;
      if (xout) xout[i] = (T)xi;
    }
  }
}

// r = f - A_L xw, summed in FP64 and stored in FP32 for the product with X
// (xw = null: r = f); one conversion per row instead of one per product.
template <typename T>
__global__ void k_dense_resid(int m, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                              const double *__restrict__ val, const T *__restrict__ f, const double *__restrict__ xw,
                              float *__restrict__ r, const KState *st) {
  if (is_done(st)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double s = to_f64(f[i]);
  if (xw)
    for (int e = rp[i]; e < rp[i + 1]; ++e) s = __fma_rn(-val[e], xw[ci[e]], s);
  r[i] = f64_to_f32(s);
}

// x = X f refined `steps` times: xw += X (f - A_L xw).
template <typename T>
amg_status dense_refined_solve(amg_hierarchy *h, const T *f, T *x, int steps, cudaStream_t s, const KState *st) {
  const Level &c = h->lev[h->L];
  const int m = c.n;
  float *r = (float *)h->dense_r;
  double *xw = h->dense_r + (m + AMG_PAD);
  const int grid = grid_for((long long)m * 32, AMG_THREADS);
  for (int k = 0; k <= steps; ++k) {
    k_dense_resid<T><<<cdiv(m, AMG_THREADS), AMG_THREADS, 0, s>>>(m, c.rp, c.ci, c.val, f, k ? xw : nullptr, r,
                                                                 st);
    count_launch();
    k_gemv32<float, T><<<grid, AMG_THREADS, 0, s>>>(m, h->ainv32, r, xw, k ? 1 : 0, k == steps ? x : nullptr, st);
    count_launch();
  }
  return amg_cuda_status(cudaGetLastError());
}
template amg_status dense_refined_solve<double>(amg_hierarchy *, const double *, double *, int, cudaStream_t,
                                                const KState *);
template amg_status dense_refined_solve<float>(amg_hierarchy *, const float *, float *, int, cudaStream_t,
                                               const KState *);

// ---------------------------------------------------------------------------
// Coarsest solve: Jacobi-PCG to ||r|| <= 1e-12 ||f|| (max 1000 iterations) in
// the pipelined arrangement, so the three inner products of an iteration
// come from vectors known before its matrix product: one persistent
// cooperative kernel per solve, one bounded software grid barrier per
// iteration.
//
// Block b owns the rows of a contiguous range holding about nnz/G entries.
// Setup sorts each block's rows by length once (stable, so the order is
// fixed); the kernel keeps the state of its rows (ten vectors and 1/a_ii)
// in shared memory, in that order, and stages its matrix slice as SELL-32
// (slices of 32 lanes, entry q of a lane at slice offset + 32 q; Kreutzer et
// al., SIAM J. Sci. Comput. 36(5), 2014): rows up to 16 entries take one
// lane, up to 64 entries four lanes, up to 256 sixteen lanes; longer rows
// take a warp and are read from global memory.  A lane gathers all of its
// (at most 16) neighbours in one round, and a warp runs exactly as many FMAs
// as its longest lane needs: FP64 instructions cost the full pipe time even
// for inactive lanes, so the FMA count is chosen by a warp-uniform branch
// rather than by predication.  The only global traffic of an iteration is the
// halo vector m: written by owners, gathered once per nonzero.
// ---------------------------------------------------------------------------
#define CG_RTOL 1e-12
#define CG_MAXIT 1000
#define CG_KEYS 258     // sort keys: row length 0..256, 257 for longer rows
#ifndef CG_MAXQ
#define CG_MAXQ 16      // neighbours a lane gathers in one round
#endif


__device__ __forceinline__ int cg_key(int len) { return len < CG_KEYS - 1 ? len : CG_KEYS - 1; }

// Time of a row per CG iteration relative to one of its entries: measured
// per block on GB300, an iteration costs about 2.6 clocks per entry (the
// SpMV) and 8 per row (vector updates and inner products).
#define CG_ROW_COST 3

// Smallest row r whose work prefix rp[r] + CG_ROW_COST r reaches target.
__device__ __forceinline__ int cg_first_row_with(const int32_t *rp, int n, long long target) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((long long)rp[mid] + (long long)CG_ROW_COST * mid >= target) hi = mid; else lo = mid + 1;
  }
  return lo;
}

// One warp per block of the coarse CG grid: the block's row range (about
// 1/G of the FP64 work) and its rows sorted by length, stable.  meta[5 b ..] =
// first row, end of the 1-lane rows (<= 16 entries), end of the 4-lane rows
// (<= 64), end of the 16-lane rows (<= 256), end of the range.
__global__ void k_cg_prepare(int n, const int32_t *__restrict__ rp, int *__restrict__ ord, int *__restrict__ meta) {
  __shared__ int cnt[CG_KEYS];
  const int lane = threadIdx.x, b = blockIdx.x, G = gridDim.x;
  const long long work = (long long)rp[n] + (long long)CG_ROW_COST * n;
  const int r0 = b == 0 ? 0 : cg_first_row_with(rp, n, work * b / G);
  const int r1 = b + 1 == G ? n : cg_first_row_with(rp, n, work * (b + 1) / G);
  for (int k = lane; k < CG_KEYS; k += 32) cnt[k] = 0;
  __syncwarp();
  for (int i = r0 + lane; i < r1; i += 32) atomicAdd(&cnt[cg_key(rp[i + 1] - rp[i])], 1);
  __syncwarp();
  if (lane == 0) {
    int s = 0, e1 = 0, e2 = 0, e3 = 0;
    for (int k = 0; k < CG_KEYS; ++k) {
      const int c = cnt[k];
      cnt[k] = s;
      s += c;
      if (k == 16) e1 = s;
      if (k == 64) e2 = s;
      if (k == 256) e3 = s;
    }
    meta[5 * b + 0] = r0;
    meta[5 * b + 1] = r0 + e1;
    meta[5 * b + 2] = r0 + e2;
    meta[5 * b + 3] = r0 + e3;
    meta[5 * b + 4] = r1;
  }
  __syncwarp();
  // stable scatter: rows in index order, equal keys ranked by lane
  for (int base = r0; base < r1; base += 32) {
    const int i = base + lane;
    const bool valid = i < r1;
    const int key = valid ? cg_key(rp[i + 1] - rp[i]) : -1;
    const unsigned same = __match_any_sync(0xffffffffu, key);
    const int rank = __popc(same & ((1u << lane) - 1u));
    if (valid) ord[r0 + cnt[key] + rank] = i;
    __syncwarp();
    if (valid && rank == 0) cnt[key] += __popc(same);
    __syncwarp();
  }
}

// Partial row sum of one lane: entries q = 0..N-1 at cols[q * stride], of
// which the first `cnt` exist; w continues the lane's FMA chain.  From four
// entries on, even and odd entries form two chains (halving the dependent
// FP64 latency) that meet at the end.
template <int N>
__device__ __forceinline__ double cg_lane_dot(const int *cols, const double *vals, int stride, int cnt,
                                              const double *u, double w) {
  double vv[N], uu[N];
#pragma unroll
  for (int q = 0; q < N; ++q) {
    const bool in = q < cnt;
    const int c = in ? cols[q * stride] : 0;
    vv[q] = in ? vals[q * stride] : 0.0;
    uu[q] = in ? __ldcg(&u[c]) : 0.0;
  }
  if (N < 4) {
#pragma unroll
    for (int q = 0; q < N; ++q) w = __fma_rn(vv[q], uu[q], w);
    return w;
  }
  double w1 = 0.0;
#pragma unroll
  for (int q = 0; q < N; q += 2) {
    w = __fma_rn(vv[q], uu[q], w);
    if (q + 1 < N) w1 = __fma_rn(vv[q + 1], uu[q + 1], w1);
  }
  return __dadd_rn(w, w1);
}

// Dispatch on the warp's largest lane count (warp-uniform): exactly that many
// FMAs per lane, or rounds of CG_MAXQ for longer rows.
__device__ __forceinline__ double cg_row_part(const int *cols, const double *vals, int stride, int cnt, int wmax,
                                              const double *u) {
  switch (wmax) {
    case 0: return 0.0;
    case 1: return cg_lane_dot<1>(cols, vals, stride, cnt, u, 0.0);
    case 2: return cg_lane_dot<2>(cols, vals, stride, cnt, u, 0.0);
    case 3: return cg_lane_dot<3>(cols, vals, stride, cnt, u, 0.0);
    case 4: return cg_lane_dot<4>(cols, vals, stride, cnt, u, 0.0);
    case 5: return cg_lane_dot<5>(cols, vals, stride, cnt, u, 0.0);
    case 6: return cg_lane_dot<6>(cols, vals, stride, cnt, u, 0.0);
    case 7: return cg_lane_dot<7>(cols, vals, stride, cnt, u, 0.0);
    case 8: return cg_lane_dot<8>(cols, vals, stride, cnt, u, 0.0);
#if CG_MAXQ >= 16
    case 9: return cg_lane_dot<9>(cols, vals, stride, cnt, u, 0.0);
    case 10: return cg_lane_dot<10>(cols, vals, stride, cnt, u, 0.0);
    case 11: return cg_lane_dot<11>(cols, vals, stride, cnt, u, 0.0);
    case 12: return cg_lane_dot<12>(cols, vals, stride, cnt, u, 0.0);
    case 13: return cg_lane_dot<13>(cols, vals, stride, cnt, u, 0.0);
    case 14: return cg_lane_dot<14>(cols, vals, stride, cnt, u, 0.0);
    case 15: return cg_lane_dot<15>(cols, vals, stride, cnt, u, 0.0);
    case 16: return cg_lane_dot<16>(cols, vals, stride, cnt, u, 0.0);
#endif
    default: {
      double w = 0.0;
      for (int q0 = 0; q0 < wmax; q0 += CG_MAXQ)
        w = cg_lane_dot<CG_MAXQ>(cols + (size_t)q0 * stride, vals + (size_t)q0 * stride, stride, cnt - q0, u, w);
      return w;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(CG_THREADS, 1)
    k_coarse_cg(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const double *__restrict__ val,
                const double *__restrict__ dinv, const T *__restrict__ f, T *__restrict__ xout, CoarseCG cg,
                const KState *st, unsigned *eflags) {
  if (is_done(st)) return;
  extern __shared__ __align__(16) unsigned char cg_smem[];
  __shared__ double red_w[3][CG_THREADS];  // block reduction, one row per inner product
  __shared__ double tot_sh[3];
  __shared__ int fail_sh;
  __shared__ int gs[5], nslice_sh[4], wl_sh[CG_THREADS / 32 + 1];
  __shared__ long long sell_total_sh;
  const unsigned G = gridDim.x;
  const int nwarps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int *meta = cg.meta + 5 * blockIdx.x;
  const int P0 = meta[0], nr = meta[4] - P0;
  // group g (0..3) holds positions [gs[g], gs[g+1]) with lanes_of(g) lanes per row
  if (threadIdx.x < 5) gs[threadIdx.x] = threadIdx.x == 0 ? 0 : meta[threadIdx.x] - P0;
  __syncthreads();
  auto lanes_of = [](int g) { return g == 3 ? 32 : 1 << (2 * g); };
  auto log_lanes = [](int g) { return g == 3 ? 5 : 2 * g; };
  // dynamic shared memory, in order of priority:
  //   [row ids: nr][row lengths: nr][state r,u,w,m,n,z,q,s,p,x,d: 11 nr doubles]
  //   [slice offsets: ns + 1][warp of each slice: ns][slices by warp: ns]
  //   [SELL columns][SELL values]
  const size_t ids_bytes = (size_t)nr * 8;
  const size_t st_off = (ids_bytes + 15) / 16 * 16;
  const size_t sl_off = st_off + (size_t)nr * 8 * (CG_STATE + 1);
  int ns_abc = 0;
  for (int g = 0; g < 3; ++g) ns_abc += (gs[g + 1] - gs[g] + (32 / lanes_of(g)) - 1) / (32 / lanes_of(g));
  const size_t sell_off = (sl_off + (size_t)(3 * ns_abc + 1) * 4 + 15) / 16 * 16;
  const bool local_ids = ids_bytes <= cg.smem;
  const bool local_state = sl_off <= cg.smem;
  int *s_row = (int *)cg_smem;
  int *s_len = s_row + nr;
  double *s_st = (double *)(cg_smem + st_off);
  int *s_slice = (int *)(cg_smem + sl_off);
  int *s_wsl = s_slice + ns_abc + 1;
  int *s_list = s_wsl + ns_abc;  // slice indices grouped by warp: [wl_sh[w], wl_sh[w + 1])
  if (threadIdx.x == 0) fail_sh = 0;
  if (local_ids) {
    for (int t = threadIdx.x; t < nr; t += blockDim.x) {
      const int i = cg.ord[P0 + t];
      s_row[t] = i;
      s_len[t] = rp[i + 1] - rp[i];
    }
  }
  __syncthreads();
  auto row_at = [&](int pos) { return local_ids ? s_row[pos] : cg.ord[P0 + pos]; };
  auto len_at = [&](int pos) {
    if (local_ids) return s_len[pos];
    const int i = cg.ord[P0 + pos];
    return (int)(rp[i + 1] - rp[i]);
  };
  // SELL slice offsets and the warp of each slice (thread 0; slices are few).
  // A slice costs about width + log2(lanes per row) + 3 FP64 instructions
  // (the inner products); the slices go, widest first, to the least loaded
  // warp, and each warp's slices are listed in index order.
  if (threadIdx.x == 0) {
    long long off = 0;
    int j = 0;
    const bool room = sl_off + (size_t)(3 * ns_abc + 1) * 4 <= cg.smem;
    for (int g = 0; g < 3; ++g) {
      const int rs = 32 / lanes_of(g);
      nslice_sh[g] = j;
      for (int a = gs[g]; a < gs[g + 1]; a += rs, ++j) {
        const int last = min(a + rs, gs[g + 1]) - 1;  // rows ascend by length within a group
        const int width = (len_at(last) + lanes_of(g) - 1) / lanes_of(g);
        if (room) s_slice[j] = (int)off;
        off += 32ll * width;
      }
    }
    nslice_sh[3] = j;
    if (room) {
      s_slice[j] = (int)off;
      int load[CG_THREADS / 32];
      // warps 0-2 also sum the partials of one inner product each
      for (int w = 0; w < nwarps; ++w) load[w] = w < 3 ? 12 : 0;
      for (int g = 2; g >= 0; --g)
        for (int jj = nslice_sh[g + 1] - 1; jj >= nslice_sh[g]; --jj) {
          int best = 0;
          for (int w = 1; w < nwarps; ++w)
            if (load[w] < load[best]) best = w;
          load[best] += ((s_slice[jj + 1] - s_slice[jj]) >> 5) + log_lanes(g) + 3;
          s_wsl[jj] = best;
        }
      // counts, then list starts, then the lists (load[] reused as cursors)
      for (int w = 0; w < nwarps; ++w) load[w] = 0;
      for (int jj = 0; jj < j; ++jj) ++load[s_wsl[jj]];
      int acc = 0;
      for (int w = 0; w < nwarps; ++w) {
        wl_sh[w] = acc;
        acc += load[w];
        load[w] = wl_sh[w];
      }
      wl_sh[nwarps] = acc;
      for (int jj = 0; jj < j; ++jj) s_list[load[s_wsl[jj]]++] = jj;
    }
    sell_total_sh = room ? off : -1;
  }
  __syncthreads();
  const long long sell_n = sell_total_sh;
  const size_t sell_val_off = sell_off + ((size_t)(sell_n > 0 ? sell_n : 0) * 4 + 15) / 16 * 16;
  const bool staged = local_state && sell_n >= 0 && sell_val_off + (size_t)sell_n * 8 <= cg.smem;
  int *sell_ci = (int *)(cg_smem + sell_off);
  double *sell_val = (double *)(cg_smem + sell_val_off);
  auto group_of = [&](int j) { return j < nslice_sh[1] ? 0 : j < nslice_sh[2] ? 1 : 2; };
  if (staged) {
    // warp per slice: entry q of lane l is entry sub + LN q of the lane's row
    for (int j = warp; j < nslice_sh[3]; j += nwarps) {
      const int g = group_of(j), ln = lanes_of(g), rs = 32 / ln;
      const int pos = gs[g] + (j - nslice_sh[g]) * rs + lane / ln, sub = lane % ln;
      const bool valid = pos < gs[g + 1];
      const int i = valid ? row_at(pos) : 0;
      const int L = valid ? len_at(pos) : 0;
      const int b = valid ? rp[i] : 0;
      const int width = (s_slice[j + 1] - s_slice[j]) >> 5;
      for (int q = 0; q < width; ++q) {
        const int e = sub + ln * q;
        if (e < L) {
          sell_ci[s_slice[j] + 32 * q + lane] = ci[b + e];
          sell_val[s_slice[j] + 32 * q + lane] = val[b + e];
        }
      }
    }
  }
  __syncthreads();
  // row state by position: in shared memory, or in the global work vectors
  // (vector k of the row at position t at sbase[k * sstride + t])
  double *const sbase = local_state ? s_st : cg.state + P0;
  const size_t sstride = local_state ? (size_t)nr : (size_t)n + AMG_PAD;
#define CGV(k) (sbase + (size_t)(k) * sstride)
  double *vr = CGV(0), *vu = CGV(1), *vw = CGV(2), *vm = CGV(3), *vn = CGV(4);
  double *vz = CGV(5), *vq = CGV(6), *vs = CGV(7), *vp = CGV(8), *vx = CGV(9);
#undef CGV
  // published vector (u for the first product, then m = D^-1 w), double
  // buffered by iteration parity: a block may publish the next one while
  // another still reads the current one
  double *pub[2] = {cg.halo[0], cg.halo[1]};
  auto dinv_at = [&](int t) { return local_state ? s_st[(size_t)10 * nr + t] : __ldg(&dinv[row_at(t)]); };
  GridBarrier gb{cg.bar, 0u};
  // Block partials of (r,u), (w,u), (r,r): every FP64 warp instruction costs
  // the same whatever the number of active lanes, so the values are halved in
  // shared memory by whole warps and the last 32 of each product go to their
  // own warp; lane 0 of warps 0-2 publishes the block's three partials.
  auto block_partials = [&](double (&v)[3], double *part) {
    const int t = threadIdx.x;
    red_w[0][t] = v[0];
    red_w[1][t] = v[1];
    red_w[2][t] = v[2];
    __syncthreads();
    for (int h = blockDim.x >> 1; h >= 32; h >>= 1) {
      if (t < h) {
        red_w[0][t] += red_w[0][t + h];
        red_w[1][t] += red_w[1][t + h];
        red_w[2][t] += red_w[2][t + h];
      }
      __syncthreads();
    }
    if (warp < 3) {
      const double bsum = warp_sum(red_w[warp][lane]);
      if (lane == 0) part[warp * AMG_MAX_BLOCKS + blockIdx.x] = bsum;
    }
  };
  // y = A v for the block's rows into vy, each warp taking its slices; warps
  // 0-2 first issue the loads of the G partials of one inner product each
  // (kept in registers across the product, so their latency is hidden) and
  // afterwards sum them in index order per lane and a fixed shuffle tree.
  constexpr int PQ = 5;  // partials per lane loaded ahead (grids up to 160 blocks)
  auto spmv = [&](const double *v, double *vy, const double *part, bool with_totals) {
    double pa[PQ];
    const double *pk = part + (warp < 3 ? warp : 0) * AMG_MAX_BLOCKS;
    if (with_totals && warp < 3) {
#pragma unroll
      for (int q = 0; q < PQ; ++q) {
        const unsigned k = lane + 32 * q;
        pa[q] = k < G ? __ldcg(&pk[k]) : 0.0;
      }
    }
    auto slice = [&](int g, int js) {
      const int ln = lanes_of(g), rs = 32 / ln;
      const int pos = gs[g] + js * rs + lane / ln, sub = lane % ln;
      const bool valid = pos < gs[g + 1];
      const int i = valid ? row_at(pos) : 0;
      const int L = valid ? len_at(pos) : 0;
      const int cnt = L > sub ? (L - sub + ln - 1) / ln : 0;
      const int wmax = __reduce_max_sync(0xffffffffu, cnt);
      const int *cols;
      const double *vals;
      int stride;
      if (staged && g < 3) {
        const int o = s_slice[nslice_sh[g] + js] + lane;
        cols = sell_ci + o;
        vals = sell_val + o;
        stride = 32;
      } else {
        const int b = valid ? rp[i] : 0;
        cols = ci + b + sub;
        vals = val + b + sub;
        stride = ln;
      }
      double yi = cg_row_part(cols, vals, stride, cnt, wmax, v);
      for (int o = ln >> 1; o > 0; o >>= 1) yi += __shfl_xor_sync(0xffffffffu, yi, o);
      if (valid && sub == 0) vy[pos] = yi;
    };
    if (staged) {
      for (int k = wl_sh[warp]; k < wl_sh[warp + 1]; ++k) {
        const int j = s_list[k], g = group_of(j);
        slice(g, j - nslice_sh[g]);
      }
    } else {
      for (int g = 0; g < 3; ++g) {
        const int nsl = nslice_sh[g + 1] - nslice_sh[g];
        for (int js = warp; js < nsl; js += nwarps) slice(g, js);
      }
    }
    for (int js = warp; js < gs[4] - gs[3]; js += nwarps) slice(3, js);  // rows over 256 entries
    if (with_totals && warp < 3) {
      double a = 0.0;
#pragma unroll
      for (int q = 0; q < PQ; ++q)
        if (lane + 32 * q < G) a += pa[q];
      for (unsigned k0 = 32 * PQ; k0 < G; k0 += 32)  // larger grids
        if (k0 + lane < G) a += __ldcg(&pk[k0 + lane]);
      a = warp_sum(a);
      if (lane == 0) tot_sh[warp] = a;
    }
    __syncthreads();
  };

  // Pipelined Jacobi-PCG (Ghysels and Vanroose, SIAM J. Sci. Comput. 36(2),
  // 2014): the inner products of an iteration come from vectors known before
  // its matrix product, so one grid barrier per iteration publishes both the
  // halo vector m = D^-1 w and the partial sums, and the sums are formed while
  // the product n = A m runs.  Per iteration, after alpha and beta:
  //   z = n + beta z, q = m + beta q, s = w + beta s, p = u + beta p,
  //   x += alpha p, r -= alpha s, u -= alpha q, w -= alpha z,
  // with u = D^-1 r and w = A u holding by the recurrences.
  // initial phase: r = f, u = D^-1 f published, the other vectors zero
  for (int t = threadIdx.x; t < nr; t += blockDim.x) {
    const int i = row_at(t);
    const double fi = (double)f[i];
    const double di = __ldg(&dinv[i]);
    const double ui = __dmul_rn(fi, di);
    if (local_state) s_st[(size_t)10 * nr + t] = di;
    vr[t] = fi;
    vu[t] = ui;
    pub[1][i] = ui;
    vz[t] = 0.0;
    vq[t] = 0.0;
    vs[t] = 0.0;
    vp[t] = 0.0;
    vx[t] = 0.0;
  }
  bool ok = gb.sync(G, eflags, &fail_sh);
  if (ok) spmv(pub[1], vw, nullptr, false);  // w = A u
  else __syncthreads();
  double acc[3] = {0.0, 0.0, 0.0};
  for (int t = threadIdx.x; t < nr; t += blockDim.x) {
    const double ri = vr[t], ui = vu[t], wi = vw[t];
    const double mi = __dmul_rn(wi, dinv_at(t));
    vm[t] = mi;
    pub[0][row_at(t)] = mi;
    acc[0] = __fma_rn(ri, ui, acc[0]);
    acc[1] = __fma_rn(wi, ui, acc[1]);
    acc[2] = __fma_rn(ri, ri, acc[2]);
  }
  // scalars: thread 0 keeps the stop threshold on (r,r) and evaluates alpha
  // and beta from the totals and the reciprocals 1/gamma and 1/(gamma alpha)
  // of the previous iteration, which two other warps form while the vectors
  // are updated, so that one division stays between a reduction and the next
  // update
  __shared__ double sc[3];  // alpha, beta, stop flag (from thread 0)
  __shared__ double rcp_sh[2];  // 1/gamma and 1/(gamma alpha) of the previous iteration
  double thresh = 0.0;
  int it = 0;
  for (it = 0;; ++it) {
    double *part = cg.part + (it & 1) * 3 * AMG_MAX_BLOCKS;
    block_partials(acc, part);
    ok = gb.sync(G, eflags, &fail_sh) && ok;
    if (ok) spmv(pub[it & 1], vn, part, true);  // n = A m, totals of this iteration
    else __syncthreads();
    if (threadIdx.x == 0) {
      const double g_i = tot_sh[0], d_i = tot_sh[1], rr = tot_sh[2];
      if (it == 0) thresh = (CG_RTOL * sqrt(rr)) * (CG_RTOL * sqrt(rr));
      bool stop = !ok || fail_sh != 0 || rr <= thresh || it >= CG_MAXIT;
      double a = 0.0, b = 0.0;
      if (!stop) {
        if (it == 0) {
          a = g_i / d_i;
        } else {
          // beta = gamma_i/gamma_{i-1}, alpha = gamma_i/(delta_i - beta gamma_i/alpha_{i-1})
          b = g_i * rcp_sh[0];
          a = g_i / (d_i - g_i * g_i * rcp_sh[1]);
        }
        stop = !isfinite(a);
      }
      sc[0] = a;
      sc[1] = b;
      sc[2] = stop ? 1.0 : 0.0;
    }
    __syncthreads();
    if (sc[2] != 0.0) break;
    const double alpha = sc[0], beta = sc[1];
    // the next iteration's 1/gamma and 1/(gamma alpha), on two other warps
    // (each division is a chain of FP64 instructions on its warp's pipe)
    if (threadIdx.x == 32) rcp_sh[0] = 1.0 / tot_sh[0];
    if (threadIdx.x == 64) rcp_sh[1] = 1.0 / (tot_sh[0] * alpha);
    double *pnext = pub[(it + 1) & 1];
    acc[0] = acc[1] = acc[2] = 0.0;
    for (int t = threadIdx.x; t < nr; t += blockDim.x) {
      const double zi = __fma_rn(beta, vz[t], vn[t]);
      const double qi = __fma_rn(beta, vq[t], vm[t]);
      const double si = __fma_rn(beta, vs[t], vw[t]);
      const double pi = __fma_rn(beta, vp[t], vu[t]);
      vx[t] = __fma_rn(alpha, pi, vx[t]);
      const double ri = __fma_rn(-alpha, si, vr[t]);
      const double ui = __fma_rn(-alpha, qi, vu[t]);
      const double wi = __fma_rn(-alpha, zi, vw[t]);
      const double mi = __dmul_rn(wi, dinv_at(t));
      vz[t] = zi;
      vq[t] = qi;
      vs[t] = si;
      vp[t] = pi;
      vr[t] = ri;
      vu[t] = ui;
      vw[t] = wi;
      vm[t] = mi;
      pnext[row_at(t)] = mi;
      acc[0] = __fma_rn(ri, ui, acc[0]);
      acc[1] = __fma_rn(wi, ui, acc[1]);
      acc[2] = __fma_rn(ri, ri, acc[2]);
    }
  }
  for (int t = threadIdx.x; t < nr; t += blockDim.x) xout[row_at(t)] = (T)vx[t];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *cg.iters = it;
    atomicAdd(cg.iters_total, (unsigned long long)it);
  }
}

// ---------------------------------------------------------------------------
// Host driver
// ---------------------------------------------------------------------------
namespace {

// Per-precision views of a level: vectors of type T, matrix values of type V,
// inverse diagonal (null for the unit-diagonal scaled FP16 levels) and the
// scale factors of the FP16 mode.
template <typename T, typename V> struct Sel;
template <> struct Sel<double, double> {
  static double *f(Level &l) { return l.f; }
  static double *x(Level &l) { return l.x; }
  static double *t(Level &l) { return l.t; }
  static double *y(Level &l) { return l.y; }
  static const double *val(const Level &l) { return l.val; }
  static const double *dinv(const Level &l) { return l.dinv; }
  static const float *sig(const Level &) { return nullptr; }
  static const float *isig(const Level &) { return nullptr; }
  static const double *cval(const Level &l) { return l.cval; }
  static const double *qval(const Level &l) { return l.qval; }
  static const double *wd(const Level &l) { return l.wd; }
};
template <> struct Sel<float, float> {
  static float *f(Level &l) { return l.f32; }
  static float *x(Level &l) { return l.x32; }
  static float *t(Level &l) { return l.t32; }
  static float *y(Level &l) { return l.y32; }
  static const float *val(const Level &l) { return l.val32; }
  static const float *dinv(const Level &l) { return l.dinv32; }
  static const float *sig(const Level &) { return nullptr; }
  static const float *isig(const Level &) { return nullptr; }
  static const float *cval(const Level &l) { return l.cval32; }
  static const float *qval(const Level &l) { return l.qval32; }
  static const float *wd(const Level &l) { return l.wd32; }
};
template <> struct Sel<float, __half> {
  static float *f(Level &l) { return l.f32; }
  static float *x(Level &l) { return l.x32; }
  static float *t(Level &l) { return l.t32; }
  static float *y(Level &l) { return l.y32; }
  static const __half *val(const Level &l) { return l.val16; }
  static const float *dinv(const Level &) { return nullptr; }
  static const float *sig(const Level &l) { return l.sig; }
  static const float *isig(const Level &l) { return l.isig; }
  static const __half *cval(const Level &) { return nullptr; }
  static const __half *qval(const Level &) { return nullptr; }
  static const float *wd(const Level &) { return nullptr; }
};

inline int row_blocks(const Level &l) {
  long long warps = ((long long)l.n * l.tpr + 31) / 32;
  return grid_for(warps * 32, AMG_THREADS);
}

// Algorithmic bytes of one matrix pass (values, columns, row pointers).
inline double bytes_A(const Level &l, int vbytes) { return (double)l.nnz * (vbytes + 4) + 4.0 * (l.n + 1); }

#define DISPATCH_TPR(l, KERNEL, ...)                                                      \
  do {                                                                                    \
    int _g = row_blocks(l);                                                               \
    switch ((l).tpr) {                                                                    \
      case 1: KERNEL<1, T, V><<<_g, AMG_THREADS, 0, s>>>(__VA_ARGS__); break;             \
      case 2: KERNEL<2, T, V><<<_g, AMG_THREADS, 0, s>>>(__VA_ARGS__); break;             \
      case 4: KERNEL<4, T, V><<<_g, AMG_THREADS, 0, s>>>(__VA_ARGS__); break;             \
      case 8: KERNEL<8, T, V><<<_g, AMG_THREADS, 0, s>>>(__VA_ARGS__); break;             \
      case 16: KERNEL<16, T, V><<<_g, AMG_THREADS, 0, s>>>(__VA_ARGS__); break;           \
      default: KERNEL<32, T, V><<<_g, AMG_THREADS, 0, s>>>(__VA_ARGS__); break;           \
    }                                                                                     \
  } while (0)

// Residual t = f - A x and Jacobi sweep on a level, by its lanes-per-row
// choice (0 = TMA-staged tiles).  Kernels without a staged form use one lane.
template <typename T, typename V>
void launch_residual(amg_hierarchy *h, const Level &l, const V *val, const T *x, const T *f, T *t, cudaStream_t s,
                     const KState *st) {
  if (l.tpr == 0 && l.st_cap > 0) {
    const size_t smem = 2 * (st_val_bytes<V>(l.st_cap) + st_col_bytes(l.st_cap));
    k_rows_staged<T, V, 0><<<l.st_grid, ST_ROWS, smem, s>>>(l.n, l.rp, l.ci, val, (const T *)nullptr, T(0), x, f, t,
                                                             l.st_cap, h->eflags, st);
    return;
  }
  Level lt = l;
  if (lt.tpr == 0) lt.tpr = 1;
  DISPATCH_TPR(lt, k_residual, lt.n, lt.perm, lt.rp, lt.ci, val, x, f, t, st);
}

template <typename T, typename V>
void launch_jacobi(amg_hierarchy *h, const Level &l, const V *val, const T *dinv, T omega, const T *x, const T *f,
                   T *out, cudaStream_t s, const KState *st) {
  if (l.tpr == 0 && l.st_cap > 0) {
    const size_t smem = 2 * (st_val_bytes<V>(l.st_cap) + st_col_bytes(l.st_cap));
    k_rows_staged<T, V, 1><<<l.st_grid, ST_ROWS, smem, s>>>(l.n, l.rp, l.ci, val, dinv, omega, x, f, out, l.st_cap,
                                                             h->eflags, st);
    return;
  }
  Level lt = l;
  if (lt.tpr == 0) lt.tpr = 1;
  DISPATCH_TPR(lt, k_jacobi, lt.n, lt.perm, lt.rp, lt.ci, val, dinv, omega, x, f, out, st);
}

// Other row kernels: one lane per row when the level uses the staged form.
#define DISPATCH_ROWS(l, KERNEL, ...)           \
  do {                                          \
    Level _lr = (l);                            \
    if (_lr.tpr == 0) _lr.tpr = 1;              \
    DISPATCH_TPR(_lr, KERNEL, __VA_ARGS__);     \
  } while (0)

template <typename T>
void coarse_solve(amg_hierarchy *h, const T *f, T *x, cudaStream_t s, const KState *st) {
  Level &c = h->lev[h->L];
  const double sz = sizeof(T);
  if (h->dense && h->ainv32) {
    const double steps = h->dense_refine;
    LaunchScope ls(h, s, PK_COARSE_DENSE, h->L,
                   (1.0 + steps) * (4.0 * c.n * (double)c.n + 16.0 * c.n) + steps * (bytes_A(c, 8) + 24.0 * c.n));
    dense_refined_solve<T>(h, f, x, h->dense_refine, s, st);
    return;
  }
  if (h->dense) {
    LaunchScope ls(h, s, PK_COARSE_DENSE, h->L, 8.0 * c.n * (double)c.n + 2.0 * sz * c.n);
    k_gemv_dense<T><<<grid_for((long long)c.n * 32, AMG_THREADS), AMG_THREADS, 0, s>>>(c.n, h->ainv, f, x, st);
    return;
  }
  if (h->cg.cl.size > 0) {
    // small level: one thread block cluster (the launch error, if any, is
    // reported by the caller's cudaGetLastError)
    LaunchScope ls(h, s, PK_COARSE_CG, h->L, bytes_A(c, 8) + 10.0 * 8.0 * c.n);
    cluster_cg_launch<T>(h->cg.cl, c.n, c.rp, c.ci, c.val, c.dinv, f, x, h->cg.iters, h->cg.iters_total, st, s);
    return;
  }
  cudaMemsetAsync(h->cg.bar, 0, 2 * sizeof(unsigned), s);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(h->cg.grid);
  cfg.blockDim = dim3(h->cg.threads);
  cfg.dynamicSmemBytes = h->cg.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // bytes per CG iteration: one matrix pass plus about ten FP64 vector passes
  LaunchScope ls(h, s, PK_COARSE_CG, h->L, bytes_A(c, 8) + 10.0 * 8.0 * c.n);
  cudaLaunchKernelEx(&cfg, k_coarse_cg<T>, c.n, (const int32_t *)c.rp, (const int32_t *)c.ci, (const double *)c.val,
                     (const double *)c.dinv, f, x, h->cg, st, h->eflags);
}

// One multigrid cycle of level k on A_k x = f (Algorithm 1; W- and F-cycles
// by the coarse correction's recursion), written to out.  guess == nullptr
// starts from x = 0 as Algorithm 1 does; otherwise from *guess, which may be
// out itself (it is consumed by the first smoothing sweep).  Vectors of
// levels below L are in their level's scaling in the FP16 mode; the coarsest
// level L is never scaled and is solved, not cycled.
template <typename T, typename V>
void cycle_level(amg_hierarchy *h, int k, const T *f, const T *guess, T *out, int kind, cudaStream_t s,
                 const KState *st) {
  using S = Sel<T, V>;
  const int L = h->L;
  if (k == L) {
    coarse_solve<T>(h, f, out, s, st);
    return;
  }
  const T omega = (T)h->prm.omega;
  const int nu_pre = h->prm.nu_pre, nu_post = h->prm.nu_post;
  const double sz = sizeof(T), szv = sizeof(V);
  // matrix arrays of a host-resident level come through a staging buffer,
  // one visit (descending or ascending) at a time
  const bool staged = stage_on(h, k);
  Level l = h->lev[k];
  Level &c = h->lev[k + 1];
  T *a = S::x(l), *b = S::t(l);
  const T *dinv = S::dinv(l);
  const V *val = S::val(l);
  const double BA = bytes_A(l, (int)szv);
  if (!guess && nu_pre == 1 && nu_post == 1 && l.op_on && S::cval(l)) {
    // residual-operator form: t = C f, restriction, coarse correction,
    // out = Q x_c + wd (f + t)
    if (staged) l = stage_acquire(h, k, SET_C, s);
    {
      LaunchScope ls(h, s, PK_OP_RESIDUAL, k, BA + 2.0 * sz * l.n);
      DISPATCH_ROWS(l, k_op_residual, l.n, l.perm, l.rp, l.ci, S::cval(l), f, b, st);
    }
    if (staged) stage_release(h, k, true, s);
    {
      LaunchScope ls(h, s, PK_RESTRICT, k, (sz + 4.0) * l.n + (sz + 4.0) * c.n + 4.0);
      k_restrict<T><<<grid_for(c.n, AMG_THREADS), AMG_THREADS, 0, s>>>(c.n, l.mrp, l.mem, b, nullptr, nullptr,
                                                                        S::f(c), st);
    }
    T *xc = S::y(c);
    const T *fc = S::f(c);
    cycle_level<T, V>(h, k + 1, fc, nullptr, xc, kind, s, st);
    if (k + 1 < L && kind == AMG_CYCLE_W) cycle_level<T, V>(h, k + 1, fc, xc, xc, AMG_CYCLE_W, s, st);
    if (k + 1 < L && kind == AMG_CYCLE_F) cycle_level<T, V>(h, k + 1, fc, xc, xc, AMG_CYCLE_V, s, st);
    if (staged) l = stage_acquire(h, k, SET_Q, s);
    {
      const double BQ = (double)l.qnnz * (szv + 4.0) + 4.0 * (l.n + 1);
      LaunchScope ls(h, s, PK_OP_POST, k, BQ + 4.0 * sz * l.n + sz * c.n);
      DISPATCH_ROWS(l, k_op_post, l.n, l.perm, l.qrp, l.qci, S::qval(l), (const T *)xc, S::wd(l), f,
                    (const T *)b, out, st);
    }
    if (staged) stage_release(h, k, false, s);
    return;
  }
  if (staged) {
    l = stage_acquire(h, k, SET_A, s);
    val = S::val(l);
  }
  // presmoothing (nu_pre >= 1 sweeps), then the residual in b
  if (!guess && nu_pre == 1 && l.fuse_pre) {
    LaunchScope ls(h, s, PK_RESIDUAL, k, BA + 4.0 * sz * l.n);
    DISPATCH_ROWS(l, k_residual0, l.n, l.perm, l.rp, l.ci, val, dinv, omega, f, a, b, st);
  } else {
    if (!guess) {
      LaunchScope ls(h, s, PK_JACOBI0, k, 3.0 * sz * l.n);
      k_jacobi0<T><<<grid_for(l.n, AMG_THREADS), AMG_THREADS, 0, s>>>(l.n, f, dinv, omega, a, st);
    } else {
      LaunchScope ls(h, s, PK_JACOBI, k, BA + 4.0 * sz * l.n);
      launch_jacobi<T, V>(h, l, val, dinv, omega, guess, f, a, s, st);
    }
    for (int sw = 1; sw < nu_pre; ++sw) {
      LaunchScope ls(h, s, PK_JACOBI, k, BA + 4.0 * sz * l.n);
      launch_jacobi<T, V>(h, l, val, dinv, omega, a, f, b, s, st);
      std::swap(a, b);
    }
    LaunchScope ls(h, s, PK_RESIDUAL, k, BA + 3.0 * sz * l.n);
    launch_residual<T, V>(h, l, val, a, f, b, s, st);
  }
  if (staged) stage_release(h, k, true, s);
  // restriction f_{k+1} = P^T r
  const float *isig_c = (k + 1 < L) ? S::isig(c) : nullptr;
  {
    LaunchScope ls(h, s, PK_RESTRICT, k, (sz + 4.0) * l.n + (sz + 4.0) * c.n + 4.0);
    k_restrict<T><<<grid_for(c.n, AMG_THREADS), AMG_THREADS, 0, s>>>(c.n, l.mrp, l.mem, b, S::sig(l), isig_c,
                                                                      S::f(c), st);
  }
  // coarse correction in y_{k+1}: one cycle (V), two (W), or an F- then a
  // V-cycle (F) of level k+1, the second from the first one's result; the
  // coarsest level is solved once
  T *xc = S::y(c);
  const T *fc = S::f(c);
  cycle_level<T, V>(h, k + 1, fc, nullptr, xc, kind, s, st);
  if (k + 1 < L && kind == AMG_CYCLE_W) cycle_level<T, V>(h, k + 1, fc, xc, xc, AMG_CYCLE_W, s, st);
  if (k + 1 < L && kind == AMG_CYCLE_F) cycle_level<T, V>(h, k + 1, fc, xc, xc, AMG_CYCLE_V, s, st);
  // prolongation and postsmoothing into out
  const float *sig = S::sig(l);
  const int nc = c.n;
  T *in = a;
  T *other = b;
  if (nu_post == 0) {
    LaunchScope ls(h, s, PK_PROLONG, k, (2.0 * sz + 4.0) * l.n + sz * nc);
    k_prolong<T><<<grid_for(l.n, AMG_THREADS), AMG_THREADS, 0, s>>>(l.n, in, l.agg, xc, sig, isig_c, out, st);
    return;
  }
  if (staged) {
    l = stage_acquire(h, k, SET_A, s);
    val = S::val(l);
  }
  // curb: current iterate; spare: a free buffer distinct from out
  T *curb, *spare;
  int sweeps = nu_post;
  if (l.fuse_post) {
    T *o = (nu_post == 1) ? out : other;
    LaunchScope ls(h, s, PK_PROLONG_JACOBI, k, BA + (4.0 * sz + 4.0) * l.n + sz * nc);
    DISPATCH_ROWS(l, k_prolong_jacobi, l.n, l.perm, l.rp, l.ci, val, dinv, omega, in, l.agg, xc, sig, isig_c, f, o,
                  st);
    curb = o;
    spare = in;
    sweeps -= 1;
  } else {
    LaunchScope ls(h, s, PK_PROLONG, k, (2.0 * sz + 4.0) * l.n + sz * nc);
    k_prolong<T><<<grid_for(l.n, AMG_THREADS), AMG_THREADS, 0, s>>>(l.n, in, l.agg, xc, sig, isig_c, other, st);
    curb = other;
    spare = in;
  }
  for (int sw = 0; sw < sweeps; ++sw) {
    T *dst = (sw == sweeps - 1) ? out : spare;
    LaunchScope ls(h, s, PK_JACOBI, k, BA + 4.0 * sz * l.n);
    launch_jacobi<T, V>(h, l, val, dinv, omega, curb, f, dst, s, st);
    spare = curb;
    curb = dst;
  }
  if (staged) stage_release(h, k, false, s);
}

template <typename T, typename V>
void vcycle_levels(amg_hierarchy *h, const T *f0, T *out0, cudaStream_t s, const KState *st) {
  cycle_level<T, V>(h, 0, f0, nullptr, out0, h->prm.cycle, s, st);
}

// KERNEL names the lanes-per-row parameter TPR_.
#define DISPATCH_TPR_PLAIN(tpr_, g_, KERNEL, ...)                                     \
  do {                                                                              \
    switch (tpr_) {                                                                 \
      case 2: { constexpr int TPR_ = 2; KERNEL<<<g_, AMG_THREADS, 0, s>>>(__VA_ARGS__); break; }   \
      case 4: { constexpr int TPR_ = 4; KERNEL<<<g_, AMG_THREADS, 0, s>>>(__VA_ARGS__); break; }   \
      case 8: { constexpr int TPR_ = 8; KERNEL<<<g_, AMG_THREADS, 0, s>>>(__VA_ARGS__); break; }   \
      case 16: { constexpr int TPR_ = 16; KERNEL<<<g_, AMG_THREADS, 0, s>>>(__VA_ARGS__); break; } \
      case 32: { constexpr int TPR_ = 32; KERNEL<<<g_, AMG_THREADS, 0, s>>>(__VA_ARGS__); break; } \
      default: { constexpr int TPR_ = 1; KERNEL<<<g_, AMG_THREADS, 0, s>>>(__VA_ARGS__); break; } \
    }                                                                               \
  } while (0)

// The level-0 visit of the FP32 cycle in the residual-operator form, from the
// FP64 residual r to the FP64 result z (the output cast folded into its last
// kernel); the coarser levels run the FP32 cycle as usual.
bool level0_fp32_op(const amg_hierarchy *h) {
  const Level &l = h->lev[0];
  return h->prm.precision == AMG_FP32 && h->L > 0 && l.op_on && l.cval32 && l.qval32 && h->prm.nu_pre == 1 &&
         h->prm.nu_post == 1;
}

void cycle_level0_fp32_io64(amg_hierarchy *h, const double *r, double *z, cudaStream_t s, const KState *st) {
  using S = Sel<float, float>;
  const int L = h->L, kind = h->prm.cycle;
  const bool staged = stage_on(h, 0);
  Level l = h->lev[0];
  Level &c = h->lev[1];
  float *b = S::t(l);
  // lanes per row of the level (0, the TMA-staged form, has no operator-form kernel: one lane)
  Level lr = l;
  lr.tpr = l.tpr == 0 ? 1 : l.tpr;
  const int tpr = lr.tpr, g = row_blocks(lr);
  float *f0 = S::f(l);
  {
    LaunchScope ls(h, s, PK_CAST, 0, 12.0 * l.n);
    k_cast_scale<double, float><<<grid_for(l.n, AMG_THREADS), AMG_THREADS, 0, s>>>(l.n, r, nullptr, f0, st);
  }
  if (staged) l = stage_acquire(h, 0, SET_C, s);
  {
    LaunchScope ls(h, s, PK_OP_RESIDUAL, 0, bytes_A(l, 4) + 8.0 * l.n);
    DISPATCH_TPR_PLAIN(tpr, g, (k_op_residual<TPR_, float, float>), l.n, l.perm, l.rp, l.ci,
                       (const float *)l.cval32, (const float *)f0, b, st);
  }
  if (staged) stage_release(h, 0, true, s);
  {
    LaunchScope ls(h, s, PK_RESTRICT, 0, 8.0 * l.n + 8.0 * c.n + 4.0);
    k_restrict<float><<<grid_for(c.n, AMG_THREADS), AMG_THREADS, 0, s>>>(c.n, l.mrp, l.mem, b, nullptr, nullptr,
                                                                          S::f(c), st);
  }
  float *xc = S::y(c);
  const float *fc = S::f(c);
  cycle_level<float, float>(h, 1, fc, nullptr, xc, kind, s, st);
  if (1 < L && kind == AMG_CYCLE_W) cycle_level<float, float>(h, 1, fc, xc, xc, AMG_CYCLE_W, s, st);
  if (1 < L && kind == AMG_CYCLE_F) cycle_level<float, float>(h, 1, fc, xc, xc, AMG_CYCLE_V, s, st);
  if (staged) l = stage_acquire(h, 0, SET_Q, s);
  {
    const double BQ = (double)l.qnnz * 8.0 + 4.0 * (l.n + 1);
    LaunchScope ls(h, s, PK_OP_POST, 0, BQ + 20.0 * l.n + 4.0 * c.n);
    DISPATCH_TPR_PLAIN(tpr, g, k_op_post_out64<TPR_>, l.n, l.perm, l.qrp, l.qci, (const float *)l.qval32,
                       (const float *)xc, (const float *)l.wd32, (const float *)f0, (const float *)b, z, st);
  }
  if (staged) stage_release(h, 0, false, s);
}

}  // namespace

amg_status vcycle_run(amg_hierarchy *h, const double *r, double *z, cudaStream_t s, const KState *st) {
  if (h->prm.precision == AMG_FP64) {
    vcycle_levels<double, double>(h, r, z, s, st);
  } else if (level0_fp32_op(h)) {
    cycle_level0_fp32_io64(h, r, z, s, st);
  } else {
    Level &l0 = h->lev[0];
    const bool half = h->prm.precision == AMG_FP16_STORAGE;
    // level 0 is scaled in the FP16 mode unless it is also the coarsest level
    const float *isig0 = (half && h->L > 0) ? l0.isig : nullptr;
    int g = grid_for(l0.n, AMG_THREADS);
    {
      LaunchScope ls(h, s, PK_CAST, 0, 12.0 * l0.n);
      k_cast_scale<double, float><<<g, AMG_THREADS, 0, s>>>(l0.n, r, isig0, l0.f32, st);
    }
    if (half) vcycle_levels<float, __half>(h, l0.f32, l0.y32, s, st);
    else vcycle_levels<float, float>(h, l0.f32, l0.y32, s, st);
    {
      LaunchScope ls(h, s, PK_CAST, 0, 12.0 * l0.n);
      k_cast_scale<float, double><<<g, AMG_THREADS, 0, s>>>(l0.n, l0.y32, isig0, z, st);
    }
  }
  return amg_cuda_status(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Setup pieces owned by this file: coarsest solver and precision copies
// ---------------------------------------------------------------------------
amg_status coarse_setup(amg_hierarchy *h, cudaStream_t s) {
  const Level &c = h->lev[h->L];
  const amg_params &p = h->prm;
  const int dense_max = p.dense_max > 0 ? p.dense_max : p.coarse_max;
  h->dense = (p.coarse_solver == AMG_COARSE_DENSE) || (p.coarse_solver == AMG_COARSE_AUTO && c.n <= dense_max);
  if (h->dense) {
    if ((long long)c.n * c.n * 8 > (8ll << 30)) return AMG_ERR_UNSUPPORTED;  // > 8 GB dense factor
    return dense_inverse(h, s);
  }
  CoarseCG &cg = h->cg;
  cg.n = c.n;
  size_t vb = sizeof(double) * (c.n + AMG_PAD);
  AMG_TRY(hier_alloc(h, (void **)&cg.halo[0], vb));
  AMG_TRY(hier_alloc(h, (void **)&cg.halo[1], vb));
  AMG_TRY(hier_alloc(h, (void **)&cg.state, vb * CG_STATE));
  AMG_TRY(hier_alloc(h, (void **)&cg.part, sizeof(double) * CG_PART_DOUBLES));
  AMG_TRY(hier_alloc(h, (void **)&cg.ord, sizeof(int) * (c.n + AMG_PAD)));
  AMG_TRY(hier_alloc(h, (void **)&cg.meta, sizeof(int) * 5 * AMG_MAX_BLOCKS));
  AMG_TRY(hier_alloc(h, (void **)&cg.bar, sizeof(unsigned) * 4));
  AMG_TRY(hier_alloc(h, (void **)&cg.iters, sizeof(int) * 4));
  AMG_TRY(hier_alloc(h, (void **)&cg.iters_total, sizeof(unsigned long long)));
  AMG_CUDA(cudaMemsetAsync(cg.iters_total, 0, sizeof(unsigned long long), s));
  AMG_TRY(coarse_cg_config(c.n, &cg));
  AMG_TRY(coarse_cg_prepare(c.n, c.rp, cg, s));
  AMG_TRY(cluster_cg_config(c.n, &cg.cl));
  return AMG_OK;
}

// FP16 storage of D^-1/2 A D^-1/2: sig_i = sqrt(a_ii), isig_i = 1/sig_i,
// val16 = a_ij isig_i isig_j rounded to FP16 (computed in FP64).
__global__ void k_scale_half(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                             const double *__restrict__ val, const double *__restrict__ dinv, __half *__restrict__ val16,
                             float *__restrict__ sig, float *__restrict__ isig, unsigned *eflags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double di = dinv[i];
  if (!(di > 0.0)) { atomicOr(eflags, AMG_EFLAG_NONSYM); return; }
  const double is = sqrt(di);
  sig[i] = (float)(1.0 / is);
  isig[i] = (float)is;
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    const double v = val[e] * is * sqrt(dinv[ci[e]]);
    val16[e] = __double2half(v);
  }
}

__global__ void k_to_f32(long long n, const double *__restrict__ a, float *__restrict__ b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

static void apply_tuned(amg_hierarchy *h);

static int choose_tpr(const Level &l) {
  double avg = l.n ? (double)l.nnz / l.n : 0.0;
  if (avg <= 12.0) return 1;
  if (avg <= 24.0) return 4;
  if (avg <= 48.0) return 8;
  if (avg <= 96.0) return 16;
  return 32;
}

amg_status precision_setup(amg_hierarchy *h, cudaStream_t s) {
  const bool mixed = h->prm.precision != AMG_FP64;
  const bool half = h->prm.precision == AMG_FP16_STORAGE;
  for (int k = 0; k <= h->L; ++k) {
    Level &l = h->lev[k];
    l.tpr = choose_tpr(l);
    // Untuned forms: fusing recomputes neighbours' values, which costs FP64
    // instructions in the FP64 cycle and FP32 ones in the mixed cycles.  Measured
    // on the 256^3 anisotropic V-cycle: FP64 split 1.47 ms (fused 1.9-3.3 ms);
    // FP32 both fused 0.99 ms (split 1.04); FP16 storage fused first sweep and
    // split post-smoothing 0.96 ms (split 1.02).
    l.fuse_pre = mixed ? 1 : 0;
    l.fuse_post = (mixed && !half) ? 1 : 0;
    size_t vd = sizeof(double) * (l.n + AMG_PAD), vf = sizeof(float) * (l.n + AMG_PAD);
    if (!mixed) {
      AMG_TRY(hier_alloc(h, (void **)&l.f, vd));
      AMG_TRY(hier_alloc(h, (void **)&l.x, vd));
      AMG_TRY(hier_alloc(h, (void **)&l.t, vd));
      AMG_TRY(hier_alloc(h, (void **)&l.y, vd));
    } else {
      AMG_TRY(hier_alloc(h, (void **)&l.f32, vf));
      AMG_TRY(hier_alloc(h, (void **)&l.x32, vf));
      AMG_TRY(hier_alloc(h, (void **)&l.t32, vf));
      AMG_TRY(hier_alloc(h, (void **)&l.y32, vf));
      if (half && k < h->L) {
        // levels below the coarsest store D^-1/2 A D^-1/2 in FP16
        AMG_TRY(hier_alloc(h, (void **)&l.val16, sizeof(__half) * (l.nnz + AMG_PAD)));
        AMG_TRY(hier_alloc(h, (void **)&l.sig, vf));
        AMG_TRY(hier_alloc(h, (void **)&l.isig, vf));
        k_scale_half<<<cdiv(l.n, AMG_THREADS), AMG_THREADS, 0, s>>>(l.n, l.rp, l.ci, l.val, l.dinv, l.val16, l.sig,
                                                                     l.isig, h->eflags);
        count_launch();
      } else {
        AMG_TRY(hier_alloc(h, (void **)&l.val32, sizeof(float) * (l.nnz + AMG_PAD)));
        AMG_TRY(hier_alloc(h, (void **)&l.dinv32, vf));
        k_to_f32<<<grid_for(l.nnz, AMG_THREADS), AMG_THREADS, 0, s>>>(l.nnz, l.val, l.val32);
        k_to_f32<<<grid_for(l.n, AMG_THREADS), AMG_THREADS, 0, s>>>(l.n, l.dinv, l.dinv32);
        count_launch(2);
        if (l.op_avail) {
          // the residual-operator form's C, Q and wd rounded to FP32
          AMG_TRY(hier_alloc(h, (void **)&l.cval32, sizeof(float) * (l.nnz + AMG_PAD)));
          AMG_TRY(hier_alloc(h, (void **)&l.qval32, sizeof(float) * (l.qnnz + AMG_PAD)));
          AMG_TRY(hier_alloc(h, (void **)&l.wd32, vf));
          k_to_f32<<<grid_for(l.nnz + AMG_PAD, AMG_THREADS), AMG_THREADS, 0, s>>>(l.nnz + AMG_PAD, l.cval, l.cval32);
          k_to_f32<<<grid_for(l.qnnz + AMG_PAD, AMG_THREADS), AMG_THREADS, 0, s>>>(l.qnnz + AMG_PAD, l.qval,
                                                                                    l.qval32);
          k_to_f32<<<grid_for(l.n, AMG_THREADS), AMG_THREADS, 0, s>>>(l.n, l.wd, l.wd32);
          count_launch(3);
        }
      }
    }
  }
  if (half) {
    unsigned f = 0;
    AMG_TRY(read_eflags(h, s, &f));
    if (f & AMG_EFLAG_NONSYM) return AMG_ERR_UNSUPPORTED;  // FP16 storage needs a positive diagonal
  }
  // TMA-staged row kernels: stage capacity (largest tile) and persistent grid
  {
    int *d_max = nullptr;
    AMG_TRY(pool_alloc((void **)&d_max, sizeof(int) * 64, s));
    AMG_CUDA(cudaMemsetAsync(d_max, 0, sizeof(int) * 64, s));
    for (int k = 0; k < h->L; ++k) {
      k_tile_max<<<grid_for(cdiv(h->lev[k].n, ST_ROWS), 256, 512), 256, 0, s>>>(h->lev[k].n, h->lev[k].rp, d_max + k);
      count_launch();
    }
    int hmax[64] = {0};
    AMG_CUDA(cudaMemcpyAsync(hmax, d_max, sizeof(int) * 64, cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
    pool_free(d_max, s);
    for (int k = 0; k < h->L; ++k) {
      Level &l = h->lev[k];
      const bool f64 = h->prm.precision == AMG_FP64, f16 = h->prm.precision == AMG_FP16_STORAGE;
      const void *vp = f64 ? (const void *)l.val : f16 ? (const void *)l.val16 : (const void *)l.val32;
      const size_t vsz = f64 ? 8 : f16 ? 2 : 4;
      const int cap = hmax[k];
      const size_t smem = 2 * ((((size_t)cap + 2 * (16 / vsz)) * vsz + 127) / 128 * 128 + st_col_bytes(cap));
      if (cap <= 0 || smem > ST_SMEM_MAX || ((uintptr_t)vp & 15) || ((uintptr_t)l.ci & 15)) continue;
      int occ = 0;
      cudaError_t e;
      if (f64) {
        cudaFuncSetAttribute(k_rows_staged<double, double, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, ST_SMEM_MAX);
        cudaFuncSetAttribute(k_rows_staged<double, double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, ST_SMEM_MAX);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_rows_staged<double, double, 0>, ST_ROWS, smem);
      } else if (f16) {
        cudaFuncSetAttribute(k_rows_staged<float, __half, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, ST_SMEM_MAX);
        cudaFuncSetAttribute(k_rows_staged<float, __half, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, ST_SMEM_MAX);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_rows_staged<float, __half, 0>, ST_ROWS, smem);
      } else {
        cudaFuncSetAttribute(k_rows_staged<float, float, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, ST_SMEM_MAX);
        cudaFuncSetAttribute(k_rows_staged<float, float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, ST_SMEM_MAX);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_rows_staged<float, float, 0>, ST_ROWS, smem);
      }
      if (e != cudaSuccess || occ < 1) { cudaGetLastError(); continue; }
      l.st_cap = cap;
      l.st_grid = std::max(1, std::min(cdiv(l.n, ST_ROWS), occ * h->num_sms));
    }
  }
  // coarse levels are irregular: their row kernels visit rows by length class
  for (int k = 1; k < h->L; ++k) {
    Level &l = h->lev[k];
    AMG_TRY(hier_alloc(h, (void **)&l.perm, sizeof(int32_t) * (l.n + AMG_PAD)));
    k_level_order<<<cdiv(l.n, ORDER_WINDOW), 512, 0, s>>>(l.n, l.rp, l.perm);
    count_launch();
  }
  apply_tuned(h);
  // Krylov work vectors at level 0 (FP64 in every precision)
  const int n = h->lev[0].n;
  size_t vd = sizeof(double) * (n + AMG_PAD);
  double **vecs[] = {&h->kb, &h->kx, &h->kr, &h->kz, &h->kp, &h->kq, &h->krold, &h->ks, &h->kt, &h->krb, &h->kph, &h->ksh};
  for (double **v : vecs) AMG_TRY(hier_alloc(h, (void **)v, vd));
  AMG_TRY(hier_alloc(h, (void **)&h->part, sizeof(double) * 8 * AMG_MAX_BLOCKS));
  AMG_TRY(hier_alloc(h, (void **)&h->counter, sizeof(unsigned) * 16));
  AMG_TRY(hier_alloc(h, (void **)&h->st, sizeof(KState)));
  AMG_CUDA(cudaMemsetAsync(h->counter, 0, sizeof(unsigned) * 16, s));
  static_assert(sizeof(KState) <= 256, "KState must fit a small pinned buffer");
  h->st_host = (KState *)pinned_small_alloc();
  if (!h->st_host) return AMG_ERR_OOM;
  return amg_cuda_status(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Autotuner: per level, times the row kernels' threads-per-row choices and the
// fused / unfused variants of the first pre- and post-smoothing sweeps on the
// level's own matrix, keeps the fastest, and caches the choice by level shape
// (rows, nonzeros, precision) for every later setup in this process.
// ---------------------------------------------------------------------------
namespace {

struct TuneChoice { int tpr, fuse_pre, fuse_post, op_on; };
std::mutex g_tune_mu;
std::map<std::tuple<int, long long, int>, TuneChoice> g_tune;

template <typename T>
float time_launch(cudaStream_t s, cudaEvent_t a, cudaEvent_t b, int reps, const std::function<void()> &fn) {
  fn();  // warm-up
  float best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(a, s);
    fn();
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    best = std::min(best, ms);
  }
  return best;
}

template <typename T, typename V>
amg_status tune_levels(amg_hierarchy *h, cudaStream_t s) {
  using S = Sel<T, V>;
  cudaEvent_t ea, eb;
  AMG_CUDA(cudaEventCreate(&ea));
  AMG_CUDA(cudaEventCreate(&eb));
  const T omega = (T)h->prm.omega;
  const int reps = 3;
  for (int k = 0; k < h->L; ++k) {
    Level &l = h->lev[k];
    const V *val = S::val(l);
    const T *dinv = S::dinv(l);
    T *f = S::f(l), *x = S::x(l), *t = S::t(l), *y = S::y(l);
    const T *xc = S::y(h->lev[k + 1]);
    const float *sig = S::sig(l);
    const float *isig_c = (k + 1 < h->L) ? S::isig(h->lev[k + 1]) : nullptr;
    const double avg = l.n ? (double)l.nnz / l.n : 0.0;
    cudaMemsetAsync(f, 0, sizeof(T) * l.n, s);
    cudaMemsetAsync(x, 0, sizeof(T) * l.n, s);
    cudaMemsetAsync((void *)xc, 0, sizeof(T) * h->lev[k + 1].n, s);
    // threads per row: timed on the residual kernel
    int best_tpr = l.tpr;
    float best = 1e30f;
    const int cands[] = {0, 1, 2, 4, 8, 16, 32};
    for (int tpr : cands) {
      if (tpr == 0 && l.st_cap == 0) continue;
      if (tpr > 1 && tpr > 4.0 * avg) break;
      Level lt = l;
      lt.tpr = tpr;
      float ms = time_launch<T>(s, ea, eb, reps, [&]() { launch_residual<T, V>(h, lt, val, x, f, t, s, nullptr); });
      if (ms < best) { best = ms; best_tpr = tpr; }
    }
    l.tpr = best_tpr;
    // first presmoothing sweep: fused with the residual, or separate
    float pre_fused = time_launch<T>(s, ea, eb, reps, [&]() {
      DISPATCH_ROWS(l, k_residual0, l.n, l.perm, l.rp, l.ci, val, dinv, omega, f, x, t, (const KState *)nullptr);
    });
    float pre_split = time_launch<T>(s, ea, eb, reps, [&]() {
      k_jacobi0<T><<<grid_for(l.n, AMG_THREADS), AMG_THREADS, 0, s>>>(l.n, f, dinv, omega, x, nullptr);
      launch_residual<T, V>(h, l, val, x, f, t, s, nullptr);
    });
    l.fuse_pre = pre_fused <= pre_split ? 1 : 0;
    // prolongation: fused into the first postsmoothing sweep, or separate
    float post_fused = time_launch<T>(s, ea, eb, reps, [&]() {
      DISPATCH_ROWS(l, k_prolong_jacobi, l.n, l.perm, l.rp, l.ci, val, dinv, omega, x, l.agg, xc, sig, isig_c, f, y,
                    (const KState *)nullptr);
    });
    float post_split = time_launch<T>(s, ea, eb, reps, [&]() {
      k_prolong<T><<<grid_for(l.n, AMG_THREADS), AMG_THREADS, 0, s>>>(l.n, x, l.agg, xc, sig, isig_c, t, nullptr);
      launch_jacobi<T, V>(h, l, val, dinv, omega, t, f, y, s, nullptr);
    });
    l.fuse_post = post_fused <= post_split ? 1 : 0;
    // residual-operator form against the faster explicit forms
    if (l.op_avail && S::cval(l)) {
      float op = time_launch<T>(s, ea, eb, reps, [&]() {
        DISPATCH_ROWS(l, k_op_residual, l.n, l.perm, l.rp, l.ci, S::cval(l), f, t, (const KState *)nullptr);
        DISPATCH_ROWS(l, k_op_post, l.n, l.perm, l.qrp, l.qci, S::qval(l), xc, S::wd(l), f, (const T *)t, y,
                      (const KState *)nullptr);
      });
      l.op_on = op <= std::min(pre_fused, pre_split) + std::min(post_fused, post_split) ? 1 : 0;
    }
    count_launch(0);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[std::make_tuple(l.n, (long long)l.nnz, h->prm.precision)] =
        TuneChoice{l.tpr, l.fuse_pre, l.fuse_post, l.op_on};
  }
  cudaEventDestroy(ea);
  cudaEventDestroy(eb);
  return amg_cuda_status(cudaGetLastError());
}

}  // namespace

// Applies cached tuning choices to the levels of a new hierarchy.
static void apply_tuned(amg_hierarchy *h) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (int k = 0; k < h->L; ++k) {
    Level &l = h->lev[k];
    auto it = g_tune.find(std::make_tuple(l.n, (long long)l.nnz, h->prm.precision));
    if (it != g_tune.end()) {
      l.tpr = it->second.tpr;
      l.fuse_pre = it->second.fuse_pre;
      l.fuse_post = it->second.fuse_post;
      if (l.op_avail) l.op_on = it->second.op_on;
    }
  }
}

extern "C" amg_status amg_autotune(amg_hierarchy *h, amg_stream_t stream) {
  clear_stale_cuda_error();
  if (!h) return AMG_ERR_INVALID_ARG;
  // the tuner times device-resident kernels; tune before moving levels to the host
  if (h->residency != AMG_RESIDENT) return AMG_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  AMG_CUDA(cudaStreamSynchronize(s));
  amg_status st = h->prm.precision == AMG_FP64   ? tune_levels<double, double>(h, s)
                  : h->prm.precision == AMG_FP32 ? tune_levels<float, float>(h, s)
                                                 : tune_levels<float, __half>(h, s);
  reset_graphs(h);
  h->batch_desc_stale = 1;
  AMG_CUDA(cudaStreamSynchronize(s));
  return st;
}

extern "C" amg_status amg_level_set_config(amg_hierarchy *h, int level, int tpr, int fuse_pre, int fuse_post) {
  if (!h || level < 0 || level > h->L) return AMG_ERR_INVALID_ARG;
  if (tpr != 0 && tpr != 1 && tpr != 2 && tpr != 4 && tpr != 8 && tpr != 16 && tpr != 32) return AMG_ERR_INVALID_ARG;
  Level &l = h->lev[level];
  if (tpr == 0 && l.st_cap == 0) return AMG_ERR_UNSUPPORTED;
  l.tpr = tpr;
  l.fuse_pre = fuse_pre ? 1 : 0;
  l.fuse_post = fuse_post ? 1 : 0;
  reset_graphs(h);
  return AMG_OK;
}

extern "C" int amg_level_config(const amg_hierarchy *h, int level, int *tpr, int *fuse_pre, int *fuse_post) {
  if (!h || level < 0 || level > h->L) return -1;
  const Level &l = h->lev[level];
  if (tpr) *tpr = l.tpr;
  if (fuse_pre) *fuse_pre = l.fuse_pre;
  if (fuse_post) *fuse_post = l.fuse_post;
  return 0;
}

extern "C" int amg_level_operator_form(const amg_hierarchy *h, int level) {
  if (!h || level < 0 || level > h->L) return -1;
  return h->lev[level].op_on ? 1 : 0;
}

extern "C" amg_status amg_level_set_operator_form(amg_hierarchy *h, int level, int on) {
  if (!h || level < 0 || level > h->L) return AMG_ERR_INVALID_ARG;
  Level &l = h->lev[level];
  if (on && !l.op_avail) return AMG_ERR_UNSUPPORTED;
  l.op_on = on ? 1 : 0;
  reset_graphs(h);
  h->batch_desc_stale = 1;
  return AMG_OK;
}

// Grid, block and shared-memory configuration of the persistent coarse CG.
amg_status coarse_cg_config(int n, CoarseCG *cg) {
  int dev = 0, sms = 152, coop = 0;
  AMG_CUDA(cudaGetDevice(&dev));
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop) return AMG_ERR_UNSUPPORTED;
  AMG_CUDA(cudaFuncSetAttribute(k_coarse_cg<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, CG_SMEM_CAP));
  AMG_CUDA(cudaFuncSetAttribute(k_coarse_cg<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, CG_SMEM_CAP));
  int occ64 = 0, occ32 = 0;
  AMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ64, k_coarse_cg<double>, CG_THREADS, CG_SMEM_CAP));
  AMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ32, k_coarse_cg<float>, CG_THREADS, CG_SMEM_CAP));
  const int occ = std::min(occ64, occ32);
  if (occ < 1) return AMG_ERR_UNSUPPORTED;
  // one block per SM, at least 64 rows per block
  cg->grid = std::max(1, std::min(std::min(occ * sms, cdiv(n, 64)), AMG_MAX_BLOCKS));
  cg->threads = CG_THREADS;
  cg->smem = CG_SMEM_CAP;
  return AMG_OK;
}

// Row ranges and length order of the coarse CG blocks (cg.grid must be final).
amg_status coarse_cg_prepare(int n, const int32_t *rp, const CoarseCG &cg, cudaStream_t s) {
  if (cg.grid < 1 || cg.grid > AMG_MAX_BLOCKS || !cg.ord || !cg.meta) return AMG_ERR_INVALID_ARG;
  k_cg_prepare<<<cg.grid, 32, 0, s>>>(n, rp, cg.ord, cg.meta);
  count_launch();
  AMG_CUDA(cudaGetLastError());
  return AMG_OK;
}

// Launches the coarse CG kernel on caller-provided CSR and work memory (used by
// the allocation-free entry point); the same kernel and configuration as the
// hierarchy's coarsest solve.
amg_status coarse_cg_launch(int n, const int32_t *rp, const int32_t *ci, const double *val, const double *dinv,
                            const double *f, double *x, const CoarseCG &cg, unsigned *eflags, cudaStream_t s) {
  AMG_CUDA(cudaMemsetAsync(cg.bar, 0, 2 * sizeof(unsigned), s));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cg.grid);
  cfg.blockDim = dim3(cg.threads);
  cfg.dynamicSmemBytes = cg.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launch();
  AMG_CUDA(cudaLaunchKernelEx(&cfg, k_coarse_cg<double>, n, rp, ci, val, dinv, f, x, cg, (const KState *)nullptr,
                              eflags));
  return AMG_OK;
}

// Self-test of the bounded wait: every block waits at the grid barrier for
// one more arrival than there are blocks, so the wait must give up after
// `limit` cycles and report the timeout instead of hanging.
__global__ void k_wait_selftest(unsigned *bar, unsigned *eflags, long long limit, int *out) {
  __shared__ int fail_sh;
  if (threadIdx.x == 0) fail_sh = 0;
  __syncthreads();
  GridBarrier gb{bar, 0u};
  gb.limit = limit;
  const bool ok = gb.sync(gridDim.x + 1, eflags, &fail_sh);
  if (threadIdx.x == 0) atomicAdd(out, ok ? 0 : 1);
}

__global__ void k_selftest_convert(long long n, const double *__restrict__ in, float *__restrict__ f32,
                                   double *__restrict__ f64) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float f = f64_to_f32(in[i]);
    f32[i] = f;
    f64[i] = f32_to_f64(f);
  }
}

extern "C" amg_status amg_selftest_convert(int64_t n, const double *d_in, float *d_f32, double *d_f64,
                                           amg_stream_t stream) {
  if (n < 0 || (n > 0 && (!d_in || !d_f32 || !d_f64))) return AMG_ERR_INVALID_ARG;
  if (n == 0) return AMG_OK;
  k_selftest_convert<<<grid_for(n, AMG_THREADS), AMG_THREADS, 0, (cudaStream_t)stream>>>(n, d_in, d_f32, d_f64);
  count_launch();
  return amg_cuda_status(cudaGetLastError());
}

extern "C" amg_status amg_selftest_wait_timeout(int blocks, amg_stream_t stream) {
  if (blocks < 1 || blocks > 64) return AMG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned *buf = nullptr;
  AMG_TRY(pool_alloc((void **)&buf, 64, s));
  AMG_CUDA(cudaMemsetAsync(buf, 0, 64, s));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(64);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // all blocks resident: only the phantom is missing
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launch();
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_wait_selftest, buf, buf + 4, (long long)(1 << 22), (int *)(buf + 8));
  unsigned host[12] = {0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, buf, 48, cudaMemcpyDeviceToHost, s);
  pool_free(buf, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return amg_cuda_status(e);
  // every block must have given up and raised the timeout flag
  if ((host[4] & AMG_EFLAG_TIMEOUT) && (int)host[8] == blocks) return AMG_ERR_TIMEOUT;
  return AMG_OK;
}

extern "C" amg_status amg_vcycle(const amg_hierarchy *hc, const double *d_r, double *d_z, amg_stream_t stream) {
  clear_stale_cuda_error();
  if (!hc || !d_r || !d_z || d_r == d_z) return AMG_ERR_INVALID_ARG;
  amg_hierarchy *h = const_cast<amg_hierarchy *>(hc);
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  AMG_TRY(vcycle_run(h, d_r, d_z, s, nullptr));
  if (h->prof.on) prof_flush(h);
  unsigned f = 0;
  if (!h->dense) {
    AMG_TRY(read_eflags(h, s, &f));
    if (f & AMG_EFLAG_TIMEOUT) return AMG_ERR_TIMEOUT;
  }
  return AMG_OK;
}
