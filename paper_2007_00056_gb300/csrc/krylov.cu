// krylov.cu -- AMG-preconditioned CG (Algorithm 4), BiCGStab (Algorithm 5)
// and AMG as a stand-alone stationary solver (Sec. 3.1).
//
// The outer iteration is FP64 in every precision mode.  All scalars (alpha,
// beta, omega, rho, residual norms) live in a device KState; each reduction
// kernel finishes with a deterministic last-block sum that also evaluates the
// next scalar and the stopping test, so one iteration is a fixed launch
// sequence with no host round trip.  That sequence is captured once into a
// CUDA graph and replayed; after the stopping test fires, `done` turns every
// remaining kernel into a no-op.
#include <algorithm>
#include <cmath>

#include "common.cuh"

#define KSLOT_A 0
#define KSLOT_B 1
#define KSLOT_C 2

// ---------------------------------------------------------------------------
// Row helpers (FP64, thread-per-row or TPR lanes per row)
// ---------------------------------------------------------------------------
template <int TPR>
__device__ __forceinline__ double row_dot64(const int32_t *__restrict__ ci, const double *__restrict__ val, int b,
                                            int e, int sub, const double *__restrict__ x) {
  double s = 0.0;
  for (int k = b + sub; k < e; k += TPR) s += __ldg(&val[k]) * __ldg(&x[__ldg(&ci[k])]);
  if (TPR > 1) {
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  return s;
}

#define KROW_LOOP_BEGIN(TPR, n)                                                         \
  const int _lane = threadIdx.x & 31;                                                   \
  const int _sub = _lane & ((TPR)-1);                                                   \
  const long long _rpw = 32 / (TPR);                                                    \
  const long long _nwarps = ((long long)gridDim.x * blockDim.x) >> 5;                   \
  for (long long _base = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * _rpw; _base < (n); \
       _base += _nwarps * _rpw) {                                                       \
    const int row = (int)(_base + _lane / (TPR));                                       \
    const bool valid = row < (n);
#define KROW_LOOP_END }

// ---------------------------------------------------------------------------
// Kernels shared by both solvers
// ---------------------------------------------------------------------------
// r = b - A x; totals (b,b), (r,r) -> bnorm, rel; sets done when b = 0 or the
// start already meets the tolerance.
template <int TPR>
__global__ void k_init_residual(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                const double *__restrict__ val, const double *__restrict__ b,
                                const double *__restrict__ x, double *__restrict__ r, double *part, unsigned *counter,
                                KState *st) {
  double v[2] = {0.0, 0.0};
  KROW_LOOP_BEGIN(TPR, n)
  int rb = 0, re = 0;
  if (valid) { rb = __ldg(&rp[row]); re = __ldg(&rp[row + 1]); }
  double ax = row_dot64<TPR>(ci, val, rb, re, _sub, x);
  if (valid && _sub == 0) {
    double bi = b[row], ri = bi - ax;
    r[row] = ri;
    v[0] += bi * bi;
    v[1] += ri * ri;
  }
  KROW_LOOP_END
  double tot[2];
  if (grid_sum_last<2>(v, part, counter, tot) && threadIdx.x == 0) {
    st->bnorm = sqrt(tot[0]);
    st->rel = st->bnorm > 0.0 ? sqrt(tot[1]) / st->bnorm : 0.0;
    st->it = 0;
    st->half = 0;
    // NaN/Inf in b or x0 (or in A x0) is an invalid argument, checked first:
    // NaN compares false, so it would otherwise pass the tolerance test
    if (!isfinite(tot[0]) || !isfinite(tot[1])) { st->done = 1; st->status = AMG_ERR_INVALID_ARG; st->bnorm = 1.0; }
    else if (st->bnorm == 0.0 || st->rel <= st->rtol) { st->done = 1; st->status = AMG_OK; }
    else if (st->max_iter <= 0) { st->done = 1; st->status = AMG_ERR_NOT_CONVERGED; }
  }
}

// Residual replacement after a stop on the recurrence residual whose true
// residual misses the tolerance: r = b - A x, and the solve continues from x
// (its iteration count and limit carry on) unless r already meets rtol.
template <int TPR>
__global__ void k_restart_residual(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                   const double *__restrict__ val, const double *__restrict__ b,
                                   const double *__restrict__ x, double *__restrict__ r, double *part,
                                   unsigned *counter, KState *st) {
  double v[1] = {0.0};
  KROW_LOOP_BEGIN(TPR, n)
  int rb = 0, re = 0;
  if (valid) { rb = __ldg(&rp[row]); re = __ldg(&rp[row + 1]); }
  double ax = row_dot64<TPR>(ci, val, rb, re, _sub, x);
  if (valid && _sub == 0) {
    double ri = b[row] - ax;
    r[row] = ri;
    v[0] += ri * ri;
  }
  KROW_LOOP_END
  double tot[1];
  if (grid_sum_last<1>(v, part, counter, tot) && threadIdx.x == 0) {
    st->rel = sqrt(tot[0]) / st->bnorm;
    st->half = 0;
    if (st->rel <= st->rtol) { st->done = 1; st->status = AMG_OK; }
    else if (!isfinite(st->rel)) { st->done = 1; st->status = AMG_ERR_BREAKDOWN; }
    else if (st->it >= st->max_iter) { st->done = 1; st->status = AMG_ERR_NOT_CONVERGED; }
    else { st->done = 0; st->status = AMG_ERR_NOT_CONVERGED; }
  }
}

// ||b - A x|| / ||b|| recomputed from x (reported as rel_res_true).
template <int TPR>
__global__ void k_true_residual(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                const double *__restrict__ val, const double *__restrict__ b,
                                const double *__restrict__ x, double *part, unsigned *counter, KState *st) {
  double v[1] = {0.0};
  KROW_LOOP_BEGIN(TPR, n)
  int rb = 0, re = 0;
  if (valid) { rb = __ldg(&rp[row]); re = __ldg(&rp[row + 1]); }
  double ax = row_dot64<TPR>(ci, val, rb, re, _sub, x);
  if (valid && _sub == 0) { double ri = b[row] - ax; v[0] += ri * ri; }
  KROW_LOOP_END
  double tot[1];
  if (grid_sum_last<1>(v, part, counter, tot) && threadIdx.x == 0)
    st->rel_true = st->bnorm > 0.0 ? sqrt(tot[0]) / st->bnorm : 0.0;
}

// ---------------------------------------------------------------------------
// PCG
// ---------------------------------------------------------------------------
// p = z; rz = (r, z)
__global__ void k_pcg_start(int n, const double *__restrict__ r, const double *__restrict__ z, double *__restrict__ p,
                            double *part, unsigned *counter, KState *st) {
  if (is_done(st)) return;
  double v[1] = {0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double zi = z[i];
    p[i] = zi;
    v[0] += r[i] * zi;
  }
  double tot[1];
  if (grid_sum_last<1>(v, part, counter, tot) && threadIdx.x == 0) {
    st->rz = tot[0];
    st->xpend = 0;
    if (!isfinite(tot[0])) { st->done = 1; st->status = AMG_ERR_BREAKDOWN; }
  }
}

// q = A p; alpha = rz / (p, q)
template <int TPR>
__global__ void k_pcg_spmv(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                           const double *__restrict__ val, const double *__restrict__ p, double *__restrict__ q,
                           double *part, unsigned *counter, KState *st) {
  if (is_done(st)) return;
  double v[1] = {0.0};
  KROW_LOOP_BEGIN(TPR, n)
  int rb = 0, re = 0;
  if (valid) { rb = __ldg(&rp[row]); re = __ldg(&rp[row + 1]); }
  double ax = row_dot64<TPR>(ci, val, rb, re, _sub, p);
  if (valid && _sub == 0) { q[row] = ax; v[0] += p[row] * ax; }
  KROW_LOOP_END
  double tot[1];
  if (grid_sum_last<1>(v, part, counter, tot) && threadIdx.x == 0) {
    double pq = tot[0];
    st->pq = pq;
    if (pq == 0.0 || !isfinite(pq) || !isfinite(st->rz)) { st->done = 1; st->status = AMG_ERR_BREAKDOWN; }
    else st->alpha = st->rz / pq;
  }
}

// r -= alpha q; stopping test on ||r||.  The matching x += alpha p is
// deferred to k_pcg_xp (or to k_pcg_xfinal after the last iteration), which
// reads p anyway: x_{j+1} = x_j + alpha_j p_j either way.
__global__ void k_pcg_update(int n, double *__restrict__ r, const double *__restrict__ q, double *part,
                             unsigned *counter, KState *st) {
  if (is_done(st)) return;
  const double alpha = st->alpha;
  double v[1] = {0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    v[0] += ri * ri;
  }
  double tot[1];
  if (grid_sum_last<1>(v, part, counter, tot) && threadIdx.x == 0) {
    st->it += 1;
    st->xpend = 1;
    st->rel = sqrt(tot[0]) / st->bnorm;
    if (st->rel <= st->rtol) { st->done = 1; st->status = AMG_OK; }
    else if (!isfinite(st->rel)) { st->done = 1; st->status = AMG_ERR_BREAKDOWN; }
    else if (st->it >= st->max_iter) { st->done = 1; st->status = AMG_ERR_NOT_CONVERGED; }
  }
}

// rz_new = (r, z); beta = rz_new / rz, or, flexible, (z, r_{j+1} - r_j) / rz
// computed as -alpha (z, q) / rz, since r_{j+1} - r_j = -alpha q_j
__global__ void k_pcg_beta(int n, const double *__restrict__ r, const double *__restrict__ q,
                           const double *__restrict__ z, double *part, unsigned *counter, KState *st) {
  if (is_done(st)) return;
  const bool flex = st->flexible != 0;
  double v[2] = {0.0, 0.0};
  // two loops rather than a test inside one: a predicated-off FP64
  // instruction still costs its FP64 pipe time on this GPU
  if (flex) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      const double zi = z[i];
      v[0] += r[i] * zi;
      v[1] += zi * q[i];
    }
  } else {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[0] += r[i] * z[i];
  }
  double tot[2];
  if (grid_sum_last<2>(v, part, counter, tot) && threadIdx.x == 0) {
    double beta = (flex ? -st->alpha * tot[1] : tot[0]) / st->rz;
    if (!isfinite(beta)) { st->done = 1; st->status = AMG_ERR_BREAKDOWN; }
    st->beta = beta;
    st->rz = tot[0];
  }
}

// x += alpha p (the deferred update of this iteration), then p = z + beta p
__global__ void k_pcg_xp(int n, double *__restrict__ x, const double *__restrict__ z, double *__restrict__ p,
                         KState *st) {
  if (is_done(st)) return;
  const double alpha = st->alpha, beta = st->beta;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double pi = p[i];
    x[i] = x[i] + alpha * pi;
    p[i] = z[i] + beta * pi;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) st->xpend = 0;
}

// After the loop: the last iteration's x += alpha p when it is still pending.
__global__ void k_pcg_xfinal(int n, double *__restrict__ x, const double *__restrict__ p, const KState *st) {
  if (!st->xpend) return;
  const double alpha = st->alpha;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = x[i] + alpha * p[i];
}

// ---------------------------------------------------------------------------
// BiCGStab
// ---------------------------------------------------------------------------
// rb = r, p = r, rho = (r, r)
__global__ void k_bicg_start(int n, const double *__restrict__ r, double *__restrict__ rb, double *__restrict__ p,
                             double *part, unsigned *counter, KState *st) {
  if (is_done(st)) return;
  double v[1] = {0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double ri = r[i];
    rb[i] = ri;
    p[i] = ri;
    v[0] += ri * ri;
  }
  double tot[1];
  if (grid_sum_last<1>(v, part, counter, tot) && threadIdx.x == 0) {
    st->rho = tot[0];
    if (fabs(tot[0]) < 1e-300 || !isfinite(tot[0])) { st->done = 1; st->status = AMG_ERR_BREAKDOWN; }
  }
}

// out = A in; NV = 1: alpha = rho / (out, rb); NV = 2: omega = (out, s) / (out, out)
template <int TPR, int WHICH>
__global__ void k_bicg_spmv(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            const double *__restrict__ val, const double *__restrict__ in, double *__restrict__ out,
                            const double *__restrict__ other, double *part, unsigned *counter, KState *st) {
  if (is_done(st)) return;
  double v[2] = {0.0, 0.0};
  KROW_LOOP_BEGIN(TPR, n)
  int rb = 0, re = 0;
  if (valid) { rb = __ldg(&rp[row]); re = __ldg(&rp[row + 1]); }
  double ax = row_dot64<TPR>(ci, val, rb, re, _sub, in);
  if (valid && _sub == 0) {
    out[row] = ax;
    v[0] += ax * other[row];
    if (WHICH == 2) v[1] += ax * ax;
  }
  KROW_LOOP_END
  double tot[2];
  if (grid_sum_last<2>(v, part, counter, tot) && threadIdx.x == 0) {
    if (WHICH == 1) {
      double rv = tot[0];
      if (fabs(rv) < 1e-300 || !isfinite(rv)) { st->done = 1; st->status = AMG_ERR_BREAKDOWN; }
      else st->alpha = st->rho / rv;
    } else {
      double tt = tot[1];
      if (tt == 0.0 || !isfinite(tt)) { st->done = 1; st->status = AMG_ERR_BREAKDOWN; }
      else st->omega = tot[0] / tt;
    }
  }
}

// s = r - alpha v; half-step stopping test on ||s||
__global__ void k_bicg_s(int n, const double *__restrict__ r, const double *__restrict__ v_, double *__restrict__ s,
                         double *part, unsigned *counter, KState *st) {
  if (is_done(st)) return;
  const double alpha = st->alpha;
  double v[1] = {0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double si = r[i] - alpha * v_[i];
    s[i] = si;
    v[0] += si * si;
  }
  double tot[1];
  if (grid_sum_last<1>(v, part, counter, tot) && threadIdx.x == 0) {
    st->srel = sqrt(tot[0]) / st->bnorm;
    if (st->srel <= st->rtol) {
      st->it += 1;
      st->rel = st->srel;
      st->half = 1;  // the host applies x += alpha p~ once the loop has stopped
      st->done = 1;
      st->status = AMG_OK;
    }
  }
}

// x += alpha p~ + omega s~; r = s - omega t; stopping test; rho, beta
__global__ void k_bicg_xr(int n, double *__restrict__ x, double *__restrict__ r, const double *__restrict__ s,
                          const double *__restrict__ t, const double *__restrict__ ph, const double *__restrict__ sh,
                          const double *__restrict__ rb, double *part, unsigned *counter, KState *st) {
  if (is_done(st)) return;
  const double alpha = st->alpha, omega = st->omega;
  double v[2] = {0.0, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    x[i] = x[i] + alpha * ph[i] + omega * sh[i];
    double ri = s[i] - omega * t[i];
    r[i] = ri;
    v[0] += ri * ri;
    v[1] += ri * rb[i];
  }
  double tot[2];
  if (grid_sum_last<2>(v, part, counter, tot) && threadIdx.x == 0) {
    st->it += 1;
    st->rel = sqrt(tot[0]) / st->bnorm;
    if (st->rel <= st->rtol) { st->done = 1; st->status = AMG_OK; }
    else if (!isfinite(st->rel) || fabs(omega) < 1e-300) { st->done = 1; st->status = AMG_ERR_BREAKDOWN; }
    else if (st->it >= st->max_iter) { st->done = 1; st->status = AMG_ERR_NOT_CONVERGED; }
    else {
      double rho_new = tot[1];
      st->beta = (rho_new / st->rho) * (alpha / omega);
      st->rho = rho_new;
      if (fabs(rho_new) < 1e-300 || !isfinite(rho_new)) { st->done = 1; st->status = AMG_ERR_BREAKDOWN; }
    }
  }
}

// p = r + beta (p - omega v)
__global__ void k_bicg_p(int n, const double *__restrict__ r, const double *__restrict__ v_, double *__restrict__ p,
                         const KState *st) {
  if (is_done(st)) return;
  const double beta = st->beta, omega = st->omega;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    p[i] = r[i] + beta * (p[i] - omega * v_[i]);
}

__global__ void k_axpy_half(int n, double *__restrict__ x, const double *__restrict__ ph, const KState *st) {
  const double alpha = st->alpha;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = x[i] + alpha * ph[i];
}

// ---------------------------------------------------------------------------
// AMG as a solver: x_{j+1} = x_j + M^{-1}(b - A x_j)
// ---------------------------------------------------------------------------
// x += z
__global__ void k_amg_correct(int n, double *__restrict__ x, const double *__restrict__ z, const KState *st) {
  if (is_done(st)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = x[i] + z[i];
}

// r = b - A x recomputed from the new iterate; stopping test on ||r||
template <int TPR>
__global__ void k_amg_residual(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                               const double *__restrict__ val, const double *__restrict__ b,
                               const double *__restrict__ x, double *__restrict__ r, double *part, unsigned *counter,
                               KState *st) {
  if (is_done(st)) return;
  double v[1] = {0.0};
  KROW_LOOP_BEGIN(TPR, n)
  int rb = 0, re = 0;
  if (valid) { rb = __ldg(&rp[row]); re = __ldg(&rp[row + 1]); }
  double ax = row_dot64<TPR>(ci, val, rb, re, _sub, x);
  if (valid && _sub == 0) {
    double ri = b[row] - ax;
    r[row] = ri;
    v[0] += ri * ri;
  }
  KROW_LOOP_END
  double tot[1];
  if (grid_sum_last<1>(v, part, counter, tot) && threadIdx.x == 0) {
    st->it += 1;
    st->rel = sqrt(tot[0]) / st->bnorm;
    if (st->rel <= st->rtol) { st->done = 1; st->status = AMG_OK; }
    else if (!isfinite(st->rel)) { st->done = 1; st->status = AMG_ERR_BREAKDOWN; }
    else if (st->it >= st->max_iter) { st->done = 1; st->status = AMG_ERR_NOT_CONVERGED; }
  }
}

// ---------------------------------------------------------------------------
// Host drivers
// ---------------------------------------------------------------------------
namespace {

int vec_blocks(int n) { return grid_for(n, AMG_THREADS, 152 * 8); }
int row_blocks64(const Level &l) { return grid_for(((long long)l.n * l.tpr + 31) / 32 * 32, AMG_THREADS, 152 * 8); }

inline double spmv_bytes(const Level &l) { return (double)l.nnz * 12.0 + 4.0 * (l.n + 1) + 16.0 * l.n; }

#define KDISPATCH(l, KERNEL, ...)                                                          \
  do {                                                                                     \
    LaunchScope _ls(h, s, PK_KRYLOV_SPMV, 0, spmv_bytes(l) + 8.0 * (l).n);                 \
    int _g = row_blocks64(l);                                                              \
    switch ((l).tpr) {                                                                     \
      case 1: KERNEL<1><<<_g, AMG_THREADS, 0, s>>>(__VA_ARGS__); break;                    \
      case 4: KERNEL<4><<<_g, AMG_THREADS, 0, s>>>(__VA_ARGS__); break;                    \
      case 8: KERNEL<8><<<_g, AMG_THREADS, 0, s>>>(__VA_ARGS__); break;                    \
      case 16: KERNEL<16><<<_g, AMG_THREADS, 0, s>>>(__VA_ARGS__); break;                  \
      default: KERNEL<32><<<_g, AMG_THREADS, 0, s>>>(__VA_ARGS__); break;                  \
    }                                                                                      \
  } while (0)

#define KDISPATCH2(l, KERNEL, W, ...)                                                      \
  do {                                                                                     \
    LaunchScope _ls(h, s, PK_KRYLOV_SPMV, 0, spmv_bytes(l) + 8.0 * (l).n);                 \
    int _g = row_blocks64(l);                                                              \
    switch ((l).tpr) {                                                                     \
      case 1: KERNEL<1, W><<<_g, AMG_THREADS, 0, s>>>(__VA_ARGS__); break;                 \
      case 4: KERNEL<4, W><<<_g, AMG_THREADS, 0, s>>>(__VA_ARGS__); break;                 \
      case 8: KERNEL<8, W><<<_g, AMG_THREADS, 0, s>>>(__VA_ARGS__); break;                 \
      case 16: KERNEL<16, W><<<_g, AMG_THREADS, 0, s>>>(__VA_ARGS__); break;               \
      default: KERNEL<32, W><<<_g, AMG_THREADS, 0, s>>>(__VA_ARGS__); break;               \
    }                                                                                      \
  } while (0)

// One PCG iteration (Algorithm 4, loop body), all on stream s.
amg_status pcg_iteration(amg_hierarchy *h, cudaStream_t s) {
  Level &l = h->lev[0];
  const int n = l.n;
  KDISPATCH(l, k_pcg_spmv, n, l.rp, l.ci, l.val, h->kp, h->kq, h->part, h->counter + KSLOT_A, h->st);
  {
    LaunchScope _ls(h, s, PK_KRYLOV_VEC, 0, 3.0 * 8.0 * n);
    k_pcg_update<<<vec_blocks(n), AMG_THREADS, 0, s>>>(n, h->kr, h->kq, h->part, h->counter + KSLOT_B, h->st);
  }
  AMG_TRY(vcycle_run(h, h->kr, h->kz, s, h->st));
  {
    LaunchScope _ls(h, s, PK_KRYLOV_VEC, 0, 3.0 * 8.0 * n);
    k_pcg_beta<<<vec_blocks(n), AMG_THREADS, 0, s>>>(n, h->kr, h->kq, h->kz, h->part, h->counter + KSLOT_C, h->st);
  }
  {
    LaunchScope _ls(h, s, PK_KRYLOV_VEC, 0, 5.0 * 8.0 * n);
    k_pcg_xp<<<vec_blocks(n), AMG_THREADS, 0, s>>>(n, h->kx, h->kz, h->kp, h->st);
  }
  return amg_cuda_status(cudaGetLastError());
}

// One BiCGStab iteration (Algorithm 5, loop body).
amg_status bicg_iteration(amg_hierarchy *h, cudaStream_t s) {
  Level &l = h->lev[0];
  const int n = l.n;
  AMG_TRY(vcycle_run(h, h->kp, h->kph, s, h->st));
  KDISPATCH2(l, k_bicg_spmv, 1, n, l.rp, l.ci, l.val, h->kph, h->kq, h->krb, h->part, h->counter + KSLOT_A, h->st);
  {
    LaunchScope _ls(h, s, PK_KRYLOV_VEC, 0, 3.0 * 8.0 * n);
    k_bicg_s<<<vec_blocks(n), AMG_THREADS, 0, s>>>(n, h->kr, h->kq, h->ks, h->part, h->counter + KSLOT_B, h->st);
  }
  AMG_TRY(vcycle_run(h, h->ks, h->ksh, s, h->st));
  KDISPATCH2(l, k_bicg_spmv, 2, n, l.rp, l.ci, l.val, h->ksh, h->kt, h->ks, h->part, h->counter + KSLOT_A, h->st);
  {
    LaunchScope _ls(h, s, PK_KRYLOV_VEC, 0, 9.0 * 8.0 * n);
    k_bicg_xr<<<vec_blocks(n), AMG_THREADS, 0, s>>>(n, h->kx, h->kr, h->ks, h->kt, h->kph, h->ksh, h->krb, h->part,
                                                   h->counter + KSLOT_C, h->st);
  }
  {
    LaunchScope _ls(h, s, PK_KRYLOV_VEC, 0, 4.0 * 8.0 * n);
    k_bicg_p<<<vec_blocks(n), AMG_THREADS, 0, s>>>(n, h->kr, h->kq, h->kp, h->st);
  }
  return amg_cuda_status(cudaGetLastError());
}

// One cycle of AMG as a solver: z = M^{-1} r, x += z, r = b - A x.
amg_status amg_iteration(amg_hierarchy *h, cudaStream_t s) {
  Level &l = h->lev[0];
  const int n = l.n;
  AMG_TRY(vcycle_run(h, h->kr, h->kz, s, h->st));
  {
    LaunchScope _ls(h, s, PK_KRYLOV_VEC, 0, 3.0 * 8.0 * n);
    k_amg_correct<<<vec_blocks(n), AMG_THREADS, 0, s>>>(n, h->kx, h->kz, h->st);
  }
  KDISPATCH(l, k_amg_residual, n, l.rp, l.ci, l.val, h->kb, h->kx, h->kr, h->part, h->counter + KSLOT_A, h->st);
  return amg_cuda_status(cudaGetLastError());
}

typedef amg_status (*iter_fn)(amg_hierarchy *, cudaStream_t);

// Captures one iteration into a graph (once per hierarchy and solver).
amg_status get_graph(amg_hierarchy *h, iter_fn fn, cudaGraphExec_t *exec, long long *nodes) {
  if (*exec || !h->graphs_ok) return AMG_OK;
  cudaGraph_t g = nullptr;
  cudaStream_t cs = h->cap_stream;
  const unsigned long long before = __atomic_load_n(&g_amg_launches, __ATOMIC_RELAXED);
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    h->graphs_ok = 0;
    return AMG_OK;
  }
  amg_status st = fn(h, cs);
  cudaError_t e = cudaStreamEndCapture(cs, &g);
  // captured launches did not run: count them when the graph is replayed
  const unsigned long long after = __atomic_load_n(&g_amg_launches, __ATOMIC_RELAXED);
  *nodes = (long long)(after - before);
  count_launch(-(long long)(after - before));
  if (st != AMG_OK || e != cudaSuccess || !g) {
    cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    h->graphs_ok = 0;
    return AMG_OK;
  }
  e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *exec = nullptr;
    h->graphs_ok = 0;
  }
  return AMG_OK;
}

amg_status run_iterations(amg_hierarchy *h, iter_fn fn, cudaGraphExec_t *exec, long long *nodes, cudaStream_t s) {
  // by default a graph is captured once the hierarchy is reused: for a single
  // solve the capture and instantiation cost about what the launches they
  // replace cost; params.graphs = 1 captures on the first solve, -1 never
  // (not while host-resident levels are staged: each visit's copies are
  // issued from the host with the prediction of the next one)
  const bool use_graph = !h->prof.on && h->stg == nullptr && h->prm.graphs >= 0 &&
                         (*exec != nullptr || h->solves >= 1 || h->prm.graphs == 1);
  h->solves += 1;
  if (use_graph) AMG_TRY(get_graph(h, fn, exec, nodes));
  // enqueue a few iterations between host checks; kernels after convergence are no-ops
  int chunk = 1;
  for (;;) {
    for (int c = 0; c < chunk; ++c) {
      if (use_graph && *exec) {
        AMG_CUDA(cudaGraphLaunch(*exec, s));
        count_launch(*nodes);
      } else {
        AMG_TRY(fn(h, s));
      }
    }
    AMG_CUDA(cudaMemcpyAsync(h->st_host, h->st, sizeof(KState), cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
    if (h->prof.on) prof_flush(h);
    if (h->st_host->done) break;
    if (h->st_host->it > 100000000) return AMG_ERR_TIMEOUT;
    chunk = std::min(chunk * 2, 4);
  }
  return AMG_OK;
}

amg_status begin_solve(amg_hierarchy *h, const double *b, const double *x0, double rtol, int max_iter, int flexible,
                       cudaStream_t s) {
  const int n = h->lev[0].n;
  KState init = {};
  init.rtol = rtol;
  init.max_iter = max_iter;
  init.flexible = flexible;
  init.status = AMG_ERR_NOT_CONVERGED;
  *h->st_host = init;
  AMG_CUDA(cudaMemcpyAsync(h->st, h->st_host, sizeof(KState), cudaMemcpyHostToDevice, s));
  AMG_CUDA(cudaMemcpyAsync(h->kb, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  AMG_CUDA(cudaMemcpyAsync(h->kx, x0, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  Level &l = h->lev[0];
  KDISPATCH(l, k_init_residual, n, l.rp, l.ci, l.val, h->kb, h->kx, h->kr, h->part, h->counter + KSLOT_A, h->st);
  return amg_cuda_status(cudaGetLastError());
}

// Restarts allowed per solve after a stop whose true residual misses rtol.
#define KRYLOV_RESTARTS 4

// After a stop on the recurrence residual: computes the true residual and,
// when it misses rtol (the recurrence drifted) while iterations remain,
// replaces r by b - A x and returns true so the caller restarts the method
// from x.  At most KRYLOV_RESTARTS times per solve.
amg_status true_residual_restart(amg_hierarchy *h, cudaStream_t s, int *restarts, bool *restart) {
  const int n = h->lev[0].n;
  Level &l = h->lev[0];
  *restart = false;
  AMG_CUDA(cudaMemcpyAsync(h->st_host, h->st, sizeof(KState), cudaMemcpyDeviceToHost, s));
  AMG_CUDA(cudaStreamSynchronize(s));
  const KState k0 = *h->st_host;
  if (k0.status != AMG_OK || k0.bnorm == 0.0 || *restarts >= KRYLOV_RESTARTS || k0.it >= k0.max_iter) return AMG_OK;
  KDISPATCH(l, k_true_residual, n, l.rp, l.ci, l.val, h->kb, h->kx, h->part, h->counter + KSLOT_A, h->st);
  AMG_CUDA(cudaMemcpyAsync(h->st_host, h->st, sizeof(KState), cudaMemcpyDeviceToHost, s));
  AMG_CUDA(cudaStreamSynchronize(s));
  if (!(h->st_host->rel_true > h->st_host->rtol)) return AMG_OK;
  *restarts += 1;
  KDISPATCH(l, k_restart_residual, n, l.rp, l.ci, l.val, h->kb, h->kx, h->kr, h->part, h->counter + KSLOT_A, h->st);
  AMG_CUDA(cudaMemcpyAsync(h->st_host, h->st, sizeof(KState), cudaMemcpyDeviceToHost, s));
  AMG_CUDA(cudaStreamSynchronize(s));
  *restart = h->st_host->done == 0;
  return AMG_OK;
}

amg_status end_solve(amg_hierarchy *h, double *x, cudaStream_t s, amg_solve_info *info) {
  const int n = h->lev[0].n;
  Level &l = h->lev[0];
  AMG_CUDA(cudaMemcpyAsync(h->st_host, h->st, sizeof(KState), cudaMemcpyDeviceToHost, s));
  AMG_CUDA(cudaStreamSynchronize(s));
  if (h->st_host->bnorm == 0.0) AMG_CUDA(cudaMemsetAsync(h->kx, 0, sizeof(double) * n, s));
  KDISPATCH(l, k_true_residual, n, l.rp, l.ci, l.val, h->kb, h->kx, h->part, h->counter + KSLOT_A, h->st);
  AMG_CUDA(cudaMemcpyAsync(x, h->kx, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  AMG_CUDA(cudaMemcpyAsync(h->st_host, h->st, sizeof(KState), cudaMemcpyDeviceToHost, s));
  AMG_CUDA(cudaStreamSynchronize(s));
  if (h->prof.on) prof_flush(h);
  unsigned f = 0;
  AMG_TRY(read_eflags(h, s, &f));
  const KState &k = *h->st_host;
  amg_status status = (amg_status)k.status;
  if (f & AMG_EFLAG_TIMEOUT) status = AMG_ERR_TIMEOUT;
  if (info) {
    info->iterations = k.it;
    info->rel_res_recurrence = k.rel;
    info->rel_res_true = k.rel_true;
    info->status = status;
  }
  return status;
}

bool bad_scalar(double v) { return !(v >= 0.0) || std::isinf(v); }

}  // namespace

void reset_graphs(amg_hierarchy *h) {
  if (h->g_pcg) cudaGraphExecDestroy(h->g_pcg);
  if (h->g_bicg) cudaGraphExecDestroy(h->g_bicg);
  if (h->g_amg) cudaGraphExecDestroy(h->g_amg);
  h->g_pcg = h->g_bicg = h->g_amg = nullptr;
  h->g_pcg_nodes = h->g_bicg_nodes = h->g_amg_nodes = 0;
}

extern "C" amg_status pcg_solve(const amg_hierarchy *hc, const double *d_b, double *d_x, double rtol, int max_iter,
                                int flexible, amg_stream_t stream, amg_solve_info *info) {
  clear_stale_cuda_error();
  if (!hc || !d_b || !d_x || bad_scalar(rtol) || max_iter < 0) return AMG_ERR_INVALID_ARG;
  amg_hierarchy *h = const_cast<amg_hierarchy *>(hc);
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  const int n = h->lev[0].n;
  AMG_TRY(begin_solve(h, d_b, d_x, rtol, max_iter, flexible ? 1 : 0, s));
  int restarts = 0;
  for (bool again = true; again;) {
    AMG_TRY(vcycle_run(h, h->kr, h->kz, s, h->st));
    {
      LaunchScope _ls(h, s, PK_KRYLOV_VEC, 0, 3.0 * 8.0 * n);
      k_pcg_start<<<vec_blocks(n), AMG_THREADS, 0, s>>>(n, h->kr, h->kz, h->kp, h->part, h->counter + KSLOT_B,
                                                        h->st);
    }
    AMG_CUDA(cudaGetLastError());
    AMG_TRY(run_iterations(h, pcg_iteration, &h->g_pcg, &h->g_pcg_nodes, s));
    {
      LaunchScope _ls(h, s, PK_KRYLOV_VEC, 0, 3.0 * 8.0 * n);
      k_pcg_xfinal<<<vec_blocks(n), AMG_THREADS, 0, s>>>(n, h->kx, h->kp, h->st);
    }
    AMG_CUDA(cudaGetLastError());
    AMG_TRY(true_residual_restart(h, s, &restarts, &again));
  }
  return end_solve(h, d_x, s, info);
}

extern "C" amg_status bicgstab_solve(const amg_hierarchy *hc, const double *d_b, double *d_x, double rtol,
                                     int max_iter, amg_stream_t stream, amg_solve_info *info) {
  clear_stale_cuda_error();
  if (!hc || !d_b || !d_x || bad_scalar(rtol) || max_iter < 0) return AMG_ERR_INVALID_ARG;
  amg_hierarchy *h = const_cast<amg_hierarchy *>(hc);
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  const int n = h->lev[0].n;
  AMG_TRY(begin_solve(h, d_b, d_x, rtol, max_iter, 0, s));
  int restarts = 0;
  for (bool again = true; again;) {
    {
      LaunchScope _ls(h, s, PK_KRYLOV_VEC, 0, 4.0 * 8.0 * n);
      k_bicg_start<<<vec_blocks(n), AMG_THREADS, 0, s>>>(n, h->kr, h->krb, h->kp, h->part, h->counter + KSLOT_B,
                                                         h->st);
    }
    AMG_CUDA(cudaGetLastError());
    AMG_TRY(run_iterations(h, bicg_iteration, &h->g_bicg, &h->g_bicg_nodes, s));
    AMG_CUDA(cudaMemcpyAsync(h->st_host, h->st, sizeof(KState), cudaMemcpyDeviceToHost, s));
    AMG_CUDA(cudaStreamSynchronize(s));
    if (h->st_host->half == 1) {
      LaunchScope _ls(h, s, PK_KRYLOV_VEC, 0, 3.0 * 8.0 * n);
      k_axpy_half<<<vec_blocks(n), AMG_THREADS, 0, s>>>(n, h->kx, h->kph, h->st);
    }
    AMG_TRY(true_residual_restart(h, s, &restarts, &again));
  }
  return end_solve(h, d_x, s, info);
}

extern "C" amg_status amg_solve(const amg_hierarchy *hc, const double *d_b, double *d_x, double rtol, int max_iter,
                                amg_stream_t stream, amg_solve_info *info) {
  clear_stale_cuda_error();
  if (!hc || !d_b || !d_x || bad_scalar(rtol) || max_iter < 0) return AMG_ERR_INVALID_ARG;
  amg_hierarchy *h = const_cast<amg_hierarchy *>(hc);
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  AMG_TRY(begin_solve(h, d_b, d_x, rtol, max_iter, 0, s));
  AMG_TRY(run_iterations(h, amg_iteration, &h->g_amg, &h->g_amg_nodes, s));
  return end_solve(h, d_x, s, info);
}
