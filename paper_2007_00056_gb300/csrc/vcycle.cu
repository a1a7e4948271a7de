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

#include "common.cuh"

// ---------------------------------------------------------------------------
// Row-kernel helpers
// ---------------------------------------------------------------------------
template <typename T> struct Vec;
template <> struct Vec<double> { static __device__ __forceinline__ double ld(const double *p) { return __ldg(p); } };
template <> struct Vec<float> { static __device__ __forceinline__ float ld(const float *p) { return __ldg(p); } };

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
    const int row = (int)(_base + _lane / (TPR));                                       \
    const bool valid = row < (n);
#define ROW_LOOP_END }

// ---------------------------------------------------------------------------
// V-cycle kernels
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_jacobi0(int n, const T *__restrict__ f, const T *__restrict__ dinv, T omega, T *__restrict__ x,
                          const KState *st) {
  if (is_done(st)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    x[i] = omega * (dinv[i] * f[i]);
}

// t = f - A x
template <int TPR, typename T, typename V>
__global__ void k_residual(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
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

// xout = x + omega D^-1 (f - A x)
template <int TPR, typename T, typename V>
__global__ void k_jacobi(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                         const V *__restrict__ val, const T *__restrict__ dinv, T omega, const T *__restrict__ x,
                         const T *__restrict__ f, T *__restrict__ xout, const KState *st) {
  if (is_done(st)) return;
  ROW_LOOP_BEGIN(TPR, n)
  int b = 0, e = 0;
  if (valid) { b = __ldg(&rp[row]); e = __ldg(&rp[row + 1]); }
  T ax = row_sum<TPR, T, V>(ci, val, b, e, _sub, [&](int j) { return __ldg(&x[j]); });
  if (valid && _sub == 0) xout[row] = x[row] + omega * (dinv[row] * (f[row] - ax));
  ROW_LOOP_END
}

// Prolongation fused into the first post-smoothing sweep:
// xp = x + xc[agg]; xout = xp + omega D^-1 (f - A xp)
template <int TPR, typename T, typename V>
__global__ void k_prolong_jacobi(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                 const V *__restrict__ val, const T *__restrict__ dinv, T omega,
                                 const T *__restrict__ x, const int32_t *__restrict__ agg,
                                 const T *__restrict__ xc, const T *__restrict__ f, T *__restrict__ xout,
                                 const KState *st) {
  if (is_done(st)) return;
  ROW_LOOP_BEGIN(TPR, n)
  int b = 0, e = 0;
  if (valid) { b = __ldg(&rp[row]); e = __ldg(&rp[row + 1]); }
  T ax = row_sum<TPR, T, V>(ci, val, b, e, _sub,
                            [&](int j) { return __ldg(&x[j]) + __ldg(&xc[__ldg(&agg[j])]); });
  if (valid && _sub == 0) {
    T xp = x[row] + xc[agg[row]];
    xout[row] = xp + omega * (dinv[row] * (f[row] - ax));
  }
  ROW_LOOP_END
}

template <typename T>
__global__ void k_prolong(int n, const T *__restrict__ x, const int32_t *__restrict__ agg, const T *__restrict__ xc,
                          T *__restrict__ xout, const KState *st) {
  if (is_done(st)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    xout[i] = x[i] + xc[agg[i]];
}

// f_c[I] = sum of t over the members of I, members ascending.
template <typename T>
__global__ void k_restrict(int nc, const int32_t *__restrict__ mrp, const int32_t *__restrict__ mem,
                           const T *__restrict__ t, T *__restrict__ fc, const KState *st) {
  if (is_done(st)) return;
  for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += gridDim.x * blockDim.x) {
    int b = mrp[I], e = mrp[I + 1];
    T s = t[mem[b]];
    for (int k = b + 1; k < e; ++k) s += t[mem[k]];
    fc[I] = s;
  }
}

template <typename A, typename B>
__global__ void k_cast(int n, const A *__restrict__ a, B *__restrict__ b, const KState *st) {
  if (is_done(st)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] = (B)a[i];
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
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < m; i += warps) {
    const double *row = ainv + (size_t)i * m;
    double s = 0.0;
    for (int j = lane; j < m; j += 32) s += __ldg(&row[j]) * (double)__ldg(&f[j]);
    s = warp_sum(s);
    if (lane == 0) x[i] = (T)s;
  }
}

// ---------------------------------------------------------------------------
// Coarsest solve: Jacobi-PCG to ||r|| <= 1e-12 ||f|| (max 1000 iterations),
// one persistent cooperative kernel with a bounded software grid barrier.
// ---------------------------------------------------------------------------
#define CG_RTOL 1e-12
#define CG_MAXIT 1000
#define BARRIER_SPIN_LIMIT (1ll << 31)  // clock cycles (about one second)

struct GridSync {
  unsigned *bar;
  unsigned gen;
  bool failed;
  __device__ __forceinline__ void sync(unsigned nblocks, unsigned *eflags) {
    __syncthreads();
    if (threadIdx.x == 0 && !failed) {
      __threadfence();
      unsigned arrived = atomicAdd(&bar[0], 1u);
      if (arrived == nblocks - 1) {
        atomicExch(&bar[0], 0u);
        __threadfence();
        atomicExch(&bar[1], gen + 1);
      } else {
        long long t0 = clock64();
        while (*((volatile unsigned *)&bar[1]) == gen) {
          if (clock64() - t0 > BARRIER_SPIN_LIMIT) {
            atomicOr(eflags, AMG_EFLAG_TIMEOUT);
            failed = true;
            break;
          }
        }
      }
      __threadfence();
    }
    ++gen;
    __syncthreads();
  }
};

__device__ __forceinline__ double cg_pnew(double z, double beta, double p) { return __fma_rn(beta, p, z); }

template <typename T>
__global__ void __launch_bounds__(AMG_THREADS) k_coarse_cg(int n, const int32_t *__restrict__ rp,
                                                             const int32_t *__restrict__ ci,
                                                             const double *__restrict__ val,
                                                             const double *__restrict__ dinv, const T *__restrict__ f,
                                                             T *__restrict__ xout, CoarseCG cg, const KState *st,
                                                             unsigned *eflags) {
  if (is_done(st)) return;
  __shared__ double sh[2 * 32];
  __shared__ double red[2];
  __shared__ int failed_sh;
  const unsigned G = gridDim.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nthreads = G * blockDim.x;
  GridSync gs{cg.bar, 0u, false};
  int slot = 0;
  // reduce NV values over the grid: partials -> barrier -> everyone sums in index order
  auto grid_reduce = [&](double *v, int nv) {
    double tmp[2] = {v[0], nv > 1 ? v[1] : 0.0};
    block_sum<2>(tmp, sh);
    double *part = cg.part + slot * 2 * AMG_MAX_BLOCKS;
    if (threadIdx.x == 0) { part[blockIdx.x] = tmp[0]; part[AMG_MAX_BLOCKS + blockIdx.x] = tmp[1]; }
    gs.sync(G, eflags);
    if (threadIdx.x < 32) {
      double a = 0.0, b = 0.0;
      for (unsigned k = threadIdx.x; k < G; k += 32) { a += __ldcg(&part[k]); b += __ldcg(&part[AMG_MAX_BLOCKS + k]); }
      a = warp_sum(a);
      b = warp_sum(b);
      if (threadIdx.x == 0) { red[0] = a; red[1] = b; failed_sh = gs.failed ? 1 : 0; }
    }
    __syncthreads();
    v[0] = red[0];
    if (nv > 1) v[1] = red[1];
    slot ^= 1;
  };

  double *x = cg.x, *r = cg.r, *z = cg.z, *p = cg.p, *pn = cg.p2, *q = cg.q;
  double v[2];
  // x = 0, r = f, ||f||
  double ff = 0.0;
  for (int i = tid; i < n; i += nthreads) {
    double fi = (double)f[i];
    x[i] = 0.0;
    r[i] = fi;
    ff += fi * fi;
  }
  v[0] = ff; v[1] = 0.0;
  grid_reduce(v, 1);
  const double fnorm = sqrt(v[0]);
  int it = 0;
  if (fnorm > 0.0 && !failed_sh) {
    // z = D^-1 r, p = z
    double rz = 0.0;
    for (int i = tid; i < n; i += nthreads) {
      double ri = __ldcg(&r[i]);
      double zi = ri * __ldg(&dinv[i]);
      z[i] = zi;
      p[i] = zi;
      rz += ri * zi;
    }
    v[0] = rz;
    grid_reduce(v, 1);
    rz = v[0];
    double beta = 0.0;
    bool first = true;
    for (it = 1; it <= CG_MAXIT; ++it) {
      // phase 1: pn = z + beta p (p itself in the first iteration), q = A pn;
      // neighbours' pn are formed on the fly from z and p, which no block
      // writes in this phase
      double pq = 0.0;
      for (int i = tid; i < n; i += nthreads) {
        double s = 0.0;
        const int e1 = __ldg(&rp[i + 1]);
        for (int e = __ldg(&rp[i]); e < e1; ++e) {
          int j = __ldg(&ci[e]);
          double pj = first ? __ldcg(&p[j]) : cg_pnew(__ldcg(&z[j]), beta, __ldcg(&p[j]));
          s += __ldg(&val[e]) * pj;
        }
        double pi = first ? __ldcg(&p[i]) : cg_pnew(__ldcg(&z[i]), beta, __ldcg(&p[i]));
        pn[i] = pi;
        q[i] = s;
        pq += pi * s;
      }
      v[0] = pq;
      grid_reduce(v, 1);
      if (failed_sh) break;
      const double alpha = rz / v[0];
      // phase 2: x += alpha pn, r -= alpha q, z = D^-1 r
      double rr = 0.0, rzn = 0.0;
      for (int i = tid; i < n; i += nthreads) {
        double pi = __ldcg(&pn[i]);
        x[i] = __ldcg(&x[i]) + alpha * pi;
        double ri = __ldcg(&r[i]) - alpha * __ldcg(&q[i]);
        r[i] = ri;
        double zi = ri * __ldg(&dinv[i]);
        z[i] = zi;
        rr += ri * ri;
        rzn += ri * zi;
      }
      v[0] = rr; v[1] = rzn;
      grid_reduce(v, 2);
      if (failed_sh) break;
      double *tmp = p; p = pn; pn = tmp;
      if (sqrt(v[0]) <= CG_RTOL * fnorm) break;
      beta = v[1] / rz;
      rz = v[1];
      first = false;
    }
    if (it > CG_MAXIT) it = CG_MAXIT;
  }
  for (int i = tid; i < n; i += nthreads) xout[i] = (T)__ldcg(&x[i]);
  if (tid == 0) { *cg.iters = it; atomicAdd(cg.iters_total, (unsigned long long)it); }
}

// ---------------------------------------------------------------------------
// Host driver
// ---------------------------------------------------------------------------
namespace {

template <typename T> struct LevelVec;
template <> struct LevelVec<double> {
  static double *f(Level &l) { return l.f; }
  static double *x(Level &l) { return l.x; }
  static double *t(Level &l) { return l.t; }
  static double *y(Level &l) { return l.y; }
  static const double *val(const Level &l) { return l.val; }
  static const double *dinv(const Level &l) { return l.dinv; }
};
template <> struct LevelVec<float> {
  static float *f(Level &l) { return l.f32; }
  static float *x(Level &l) { return l.x32; }
  static float *t(Level &l) { return l.t32; }
  static float *y(Level &l) { return l.y32; }
  static const float *val(const Level &l) { return l.val32; }
  static const float *dinv(const Level &l) { return l.dinv32; }
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
      case 1: KERNEL<1, T, T><<<_g, AMG_THREADS, 0, s>>>(__VA_ARGS__); break;             \
      case 4: KERNEL<4, T, T><<<_g, AMG_THREADS, 0, s>>>(__VA_ARGS__); break;             \
      case 8: KERNEL<8, T, T><<<_g, AMG_THREADS, 0, s>>>(__VA_ARGS__); break;             \
      case 16: KERNEL<16, T, T><<<_g, AMG_THREADS, 0, s>>>(__VA_ARGS__); break;           \
      default: KERNEL<32, T, T><<<_g, AMG_THREADS, 0, s>>>(__VA_ARGS__); break;           \
    }                                                                                     \
  } while (0)

template <typename T>
void coarse_solve(amg_hierarchy *h, const T *f, T *x, cudaStream_t s, const KState *st) {
  Level &c = h->lev[h->L];
  const double sz = sizeof(T);
  if (h->dense) {
    LaunchScope ls(h, s, PK_COARSE_DENSE, h->L, 8.0 * c.n * (double)c.n + 2.0 * sz * c.n);
    k_gemv_dense<T><<<grid_for((long long)c.n * 32, AMG_THREADS), AMG_THREADS, 0, s>>>(c.n, h->ainv, f, x, st);
    return;
  }
  cudaMemsetAsync(h->cg.bar, 0, 2 * sizeof(unsigned), s);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(h->cg.grid);
  cfg.blockDim = dim3(AMG_THREADS);
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

// Runs the V-cycle below level 0 given f0 (level-0 rhs) and writes out0.
template <typename T>
void vcycle_levels(amg_hierarchy *h, const T *f0, T *out0, cudaStream_t s, const KState *st) {
  const int L = h->L;
  const T omega = (T)h->prm.omega;
  const int nu_pre = h->prm.nu_pre, nu_post = h->prm.nu_post;
  const double sz = sizeof(T);
  const T *fk[AMG_MAX_LEVELS];
  T *cur[AMG_MAX_LEVELS];
  for (int k = 0; k <= L; ++k) fk[k] = (k == 0) ? f0 : LevelVec<T>::f(h->lev[k]);
  // down sweep
  for (int k = 0; k < L; ++k) {
    Level &l = h->lev[k];
    T *a = LevelVec<T>::x(l), *b = LevelVec<T>::t(l);
    const T *dinv = LevelVec<T>::dinv(l);
    const T *val = LevelVec<T>::val(l);
    const double BA = bytes_A(l, (int)sz);
    {
      LaunchScope ls(h, s, PK_JACOBI0, k, 3.0 * sz * l.n);
      k_jacobi0<T><<<grid_for(l.n, AMG_THREADS), AMG_THREADS, 0, s>>>(l.n, fk[k], dinv, omega, a, st);
    }
    for (int sw = 1; sw < nu_pre; ++sw) {
      LaunchScope ls(h, s, PK_JACOBI, k, BA + 4.0 * sz * l.n);
      DISPATCH_TPR(l, k_jacobi, l.n, l.rp, l.ci, val, dinv, omega, a, fk[k], b, st);
      std::swap(a, b);
    }
    cur[k] = a;
    {
      LaunchScope ls(h, s, PK_RESIDUAL, k, BA + 3.0 * sz * l.n);
      DISPATCH_TPR(l, k_residual, l.n, l.rp, l.ci, val, a, fk[k], b, st);
    }
    Level &c = h->lev[k + 1];
    {
      LaunchScope ls(h, s, PK_RESTRICT, k, (sz + 4.0) * l.n + (sz + 4.0) * c.n + 4.0);
      k_restrict<T><<<grid_for(c.n, AMG_THREADS), AMG_THREADS, 0, s>>>(c.n, l.mrp, l.mem, b, LevelVec<T>::f(c), st);
    }
  }
  // coarsest
  T *xc = (L == 0) ? out0 : LevelVec<T>::y(h->lev[L]);
  coarse_solve<T>(h, fk[L], xc, s, st);
  // up sweep
  for (int k = L - 1; k >= 0; --k) {
    Level &l = h->lev[k];
    const int nc = h->lev[k + 1].n;
    T *final_out = (k == 0) ? out0 : LevelVec<T>::y(l);
    T *in = cur[k];
    T *other = (in == LevelVec<T>::x(l)) ? LevelVec<T>::t(l) : LevelVec<T>::x(l);
    const T *dinv = LevelVec<T>::dinv(l);
    const T *val = LevelVec<T>::val(l);
    const double BA = bytes_A(l, (int)sz);
    if (nu_post == 0) {
      LaunchScope ls(h, s, PK_PROLONG, k, (2.0 * sz + 4.0) * l.n + sz * nc);
      k_prolong<T><<<grid_for(l.n, AMG_THREADS), AMG_THREADS, 0, s>>>(l.n, in, l.agg, xc, final_out, st);
    } else {
      T *o = (nu_post == 1) ? final_out : other;
      {
        LaunchScope ls(h, s, PK_PROLONG_JACOBI, k, BA + (4.0 * sz + 4.0) * l.n + sz * nc);
        DISPATCH_TPR(l, k_prolong_jacobi, l.n, l.rp, l.ci, val, dinv, omega, in, l.agg, xc, fk[k], o, st);
      }
      T *pp = o, *qq = in;
      for (int sw = 1; sw < nu_post; ++sw) {
        T *dst = (sw == nu_post - 1) ? final_out : qq;
        LaunchScope ls(h, s, PK_JACOBI, k, BA + 4.0 * sz * l.n);
        DISPATCH_TPR(l, k_jacobi, l.n, l.rp, l.ci, val, dinv, omega, pp, fk[k], dst, st);
        qq = pp;
        pp = dst;
      }
    }
    xc = final_out;
  }
}

}  // namespace

amg_status vcycle_run(amg_hierarchy *h, const double *r, double *z, cudaStream_t s, const KState *st) {
  if (h->prm.precision == AMG_FP64) {
    vcycle_levels<double>(h, r, z, s, st);
  } else {
    Level &l0 = h->lev[0];
    int g = grid_for(l0.n, AMG_THREADS);
    {
      LaunchScope ls(h, s, PK_CAST, 0, 12.0 * l0.n);
      k_cast<double, float><<<g, AMG_THREADS, 0, s>>>(l0.n, r, l0.f32, st);
    }
    vcycle_levels<float>(h, l0.f32, l0.y32, s, st);
    {
      LaunchScope ls(h, s, PK_CAST, 0, 12.0 * l0.n);
      k_cast<float, double><<<g, AMG_THREADS, 0, s>>>(l0.n, l0.y32, z, st);
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
  h->dense = (p.coarse_solver == AMG_COARSE_DENSE) || (p.coarse_solver == AMG_COARSE_AUTO && c.n <= p.coarse_max);
  if (h->dense) {
    if ((long long)c.n * c.n * 8 > (8ll << 30)) return AMG_ERR_UNSUPPORTED;  // > 8 GB dense factor
    return dense_inverse(h, s);
  }
  CoarseCG &cg = h->cg;
  cg.n = c.n;
  size_t vb = sizeof(double) * (c.n + AMG_PAD);
  AMG_TRY(hier_alloc(h, (void **)&cg.x, vb));
  AMG_TRY(hier_alloc(h, (void **)&cg.r, vb));
  AMG_TRY(hier_alloc(h, (void **)&cg.z, vb));
  AMG_TRY(hier_alloc(h, (void **)&cg.p, vb));
  AMG_TRY(hier_alloc(h, (void **)&cg.p2, vb));
  AMG_TRY(hier_alloc(h, (void **)&cg.q, vb));
  AMG_TRY(hier_alloc(h, (void **)&cg.part, sizeof(double) * 4 * AMG_MAX_BLOCKS));
  AMG_TRY(hier_alloc(h, (void **)&cg.bar, sizeof(unsigned) * 4));
  AMG_TRY(hier_alloc(h, (void **)&cg.iters, sizeof(int) * 4));
  AMG_TRY(hier_alloc(h, (void **)&cg.iters_total, sizeof(unsigned long long)));
  AMG_CUDA(cudaMemsetAsync(cg.iters_total, 0, sizeof(unsigned long long), s));
  int occ64 = 0, occ32 = 0;
  AMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ64, k_coarse_cg<double>, AMG_THREADS, 0));
  AMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ32, k_coarse_cg<float>, AMG_THREADS, 0));
  int occ = std::max(1, std::min(occ64, occ32));
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device);
  if (!coop) return AMG_ERR_UNSUPPORTED;
  // a few warps of rows per block keeps the barrier wide enough but not wider
  int want = cdiv(c.n, AMG_THREADS);
  cg.grid = std::max(1, std::min(std::min(want, occ * h->num_sms), AMG_MAX_BLOCKS));
  return AMG_OK;
}

__global__ void k_to_f32(long long n, const double *__restrict__ a, float *__restrict__ b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

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
  if (h->prm.precision == AMG_FP16_STORAGE) return AMG_ERR_UNSUPPORTED;
  for (int k = 0; k <= h->L; ++k) {
    Level &l = h->lev[k];
    l.tpr = choose_tpr(l);
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
      AMG_TRY(hier_alloc(h, (void **)&l.val32, sizeof(float) * (l.nnz + AMG_PAD)));
      AMG_TRY(hier_alloc(h, (void **)&l.dinv32, vf));
      k_to_f32<<<grid_for(l.nnz, AMG_THREADS), AMG_THREADS, 0, s>>>(l.nnz, l.val, l.val32);
      k_to_f32<<<grid_for(l.n, AMG_THREADS), AMG_THREADS, 0, s>>>(l.n, l.dinv, l.dinv32);
      count_launch(2);
    }
  }
  // Krylov work vectors at level 0 (FP64 in every precision)
  const int n = h->lev[0].n;
  size_t vd = sizeof(double) * (n + AMG_PAD);
  double **vecs[] = {&h->kb, &h->kx, &h->kr, &h->kz, &h->kp, &h->kq, &h->krold, &h->ks, &h->kt, &h->krb, &h->kph, &h->ksh};
  for (double **v : vecs) AMG_TRY(hier_alloc(h, (void **)v, vd));
  AMG_TRY(hier_alloc(h, (void **)&h->part, sizeof(double) * 8 * AMG_MAX_BLOCKS));
  AMG_TRY(hier_alloc(h, (void **)&h->counter, sizeof(unsigned) * 16));
  AMG_TRY(hier_alloc(h, (void **)&h->st, sizeof(KState)));
  AMG_CUDA(cudaMemsetAsync(h->counter, 0, sizeof(unsigned) * 16, s));
  if (cudaMallocHost((void **)&h->st_host, sizeof(KState)) != cudaSuccess) { cudaGetLastError(); return AMG_ERR_OOM; }
  return amg_cuda_status(cudaGetLastError());
}

extern "C" amg_status amg_vcycle(const amg_hierarchy *hc, const double *d_r, double *d_z, amg_stream_t stream) {
  if (!hc || !d_r || !d_z || d_r == d_z) return AMG_ERR_INVALID_ARG;
  amg_hierarchy *h = const_cast<amg_hierarchy *>(hc);
  cudaStream_t s = (cudaStream_t)stream;
  AMG_TRY(vcycle_run(h, d_r, d_z, s, nullptr));
  if (h->prof.on) prof_flush(h);
  unsigned f = 0;
  if (!h->dense) {
    AMG_TRY(read_eflags(h, s, &f));
    if (f & AMG_EFLAG_TIMEOUT) return AMG_ERR_TIMEOUT;
  }
  return AMG_OK;
}
