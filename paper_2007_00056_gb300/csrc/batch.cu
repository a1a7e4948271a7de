// batch.cu -- many AMG-PCG solves in one persistent launch.
//
// Each system of the batch is owned by a team -- one thread block, or a
// thread-block cluster of 2, 4 or 8 blocks for larger systems -- that runs its
// whole flexible PCG (Algorithm 4) with the V-cycle of Algorithm 1 as
// preconditioner: every level of the hierarchy, smoothing, residual,
// restriction, dense coarsest solve and prolongation, separated by team
// barriers only (__syncthreads, or the cluster barrier).  The team size is a
// function of the system's row count alone, and every reduction is a fixed-
// order block reduction followed, in a cluster, by the sum of the blocks'
// totals in rank order read through distributed shared memory, so a system's
// iterates do not depend on which other systems share the launch: a solve in
// a batch is bitwise the solve alone.  Systems are read through per-hierarchy
// device descriptors (the levels' CSR arrays and work vectors already owned
// by each hierarchy), i.e. the batch is the block-diagonal concatenation of
// its systems without copying any of them.
#include <cooperative_groups.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace cgrp = cooperative_groups;

#define BATCH_THREADS 512
#define BATCH_MAX_COARSE 2048  // largest dense coarsest level a batched system may have

struct BatchLevel {
  int n, nc;
  const int32_t *rp, *ci;
  const void *val, *dinv;  // T-typed (double or float)
  const int32_t *agg, *mrp, *mem;
  void *f, *x, *t, *y;     // T-typed level vectors
  // residual-operator form (null when the level has none): C values (A's
  // pattern), Q = P - omega D^-1 A P in CSR, omega D^-1; T-typed
  const void *cval, *qval, *wd;
  const int32_t *qrp, *qci;
};

struct BatchSys {
  int L, n, nL;
  double omega;
  int nu_pre, nu_post;
  BatchLevel lev[AMG_MAX_LEVELS];
  const double *ainv;                      // dense inverse of the coarsest level
  const int32_t *rp0, *ci0;
  const double *val0;                      // level-0 FP64 matrix for the outer iteration
  double *r, *z, *p, *q, *rold;            // FP64 Krylov vectors
  double *f64c, *x64c;                     // FP64 coarse right-hand side / solution (FP32 mode)
};

struct BatchJob {
  const BatchSys *sys;
  const double *b;
  double *x;
};

struct BatchInfo {
  int iterations, status;
  double rel, rel_true;
};

// Team size (blocks per system) by row count: one block up to 8192 rows,
// then 2, 4 and 8 blocks, so a mid-size system is not left to one SM.
static inline int batch_team(int n) { return n <= 8192 ? 1 : n <= 24576 ? 2 : n <= 65536 ? 4 : 8; }

// ---------------------------------------------------------------------------
// block-scope helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double bsum(double v, double *sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = lane < nw ? sh[lane] : 0.0;
  s = warp_sum(s);
  return s;  // every warp computes the same total in the same order
}

// The threads of one system: C blocks of a cluster (C = 1: one block).  tid
// and nthr index the system's rows; sync() is the team barrier; sum() returns
// the same total, formed in the same order, to every thread of the team.
template <int C>
struct Team {
  int tid, nthr;
  __device__ Team() {
    const int rank = C > 1 ? (int)cgrp::this_cluster().block_rank() : 0;
    tid = rank * blockDim.x + threadIdx.x;
    nthr = C * blockDim.x;
  }
  __device__ __forceinline__ void sync() const {
    if (C > 1) cgrp::this_cluster().sync();
    else __syncthreads();
  }
  // sh: 33 doubles of the block's shared memory (sh[32] holds its total)
  __device__ double sum(double v, double *sh) const {
    const double blk = bsum(v, sh);
    if (C == 1) return blk;
    cgrp::cluster_group cl = cgrp::this_cluster();
    if (threadIdx.x == 0) sh[32] = blk;
    cl.sync();
    double tot = 0.0;
#pragma unroll
    for (int r = 0; r < C; ++r) tot += *cl.map_shared_rank(&sh[32], r);
    cl.sync();  // every block has read the totals before a later sum overwrites them
    return tot;
  }
};

template <typename T, typename V>
__device__ __forceinline__ T brow(const int32_t *rp, const int32_t *ci, const V *val, const T *x, int i) {
  T s = T(0);
  for (int e = rp[i]; e < rp[i + 1]; ++e) s += (T)val[e] * x[ci[e]];
  return s;
}

// One V-cycle of the system from a zero guess: out0 = M^{-1} f0 (level-0 vectors of type T).
// A level with the residual-operator form (Level documents C and Q) forms its
// residual as t = C f on the way down and its result as Q x_c + wd (f + t) on
// the way up; the others run the explicit sweeps.
template <typename T, int C>
__device__ void b_vcycle(const Team<C> &tm, const BatchSys &S, const T *f0, T *out0) {
  const int L = S.L;
  const T omega = (T)S.omega;
  const T *fk[AMG_MAX_LEVELS];
  T *cur[AMG_MAX_LEVELS];
  for (int k = 0; k <= L; ++k) fk[k] = k == 0 ? f0 : (const T *)S.lev[k].f;
  for (int k = 0; k < L; ++k) {
    const BatchLevel &l = S.lev[k];
    const T *val = (const T *)l.val, *dinv = (const T *)l.dinv;
    T *a = (T *)l.x, *b = (T *)l.t;
    const T *f = fk[k];
    if (l.cval) {
      const T *cv = (const T *)l.cval;
      for (int i = tm.tid; i < l.n; i += tm.nthr) b[i] = brow<T, T>(l.rp, l.ci, cv, f, i);
      tm.sync();
      cur[k] = nullptr;
      T *fc = (T *)S.lev[k + 1].f;
      for (int I = tm.tid; I < l.nc; I += tm.nthr) {
        int e0 = l.mrp[I], e1 = l.mrp[I + 1];
        T s = b[l.mem[e0]];
        for (int m = e0 + 1; m < e1; ++m) s += b[l.mem[m]];
        fc[I] = s;
      }
      tm.sync();
      continue;
    }
    for (int i = tm.tid; i < l.n; i += tm.nthr) a[i] = omega * (dinv[i] * f[i]);
    tm.sync();
    for (int sw = 1; sw < S.nu_pre; ++sw) {
      for (int i = tm.tid; i < l.n; i += tm.nthr)
        b[i] = a[i] + omega * (dinv[i] * (f[i] - brow<T, T>(l.rp, l.ci, val, a, i)));
      tm.sync();
      T *tmp = a; a = b; b = tmp;
    }
    cur[k] = a;
    for (int i = tm.tid; i < l.n; i += tm.nthr) b[i] = f[i] - brow<T, T>(l.rp, l.ci, val, a, i);
    tm.sync();
    T *fc = (T *)S.lev[k + 1].f;
    for (int I = tm.tid; I < l.nc; I += tm.nthr) {
      int e0 = l.mrp[I], e1 = l.mrp[I + 1];
      T s = b[l.mem[e0]];
      for (int m = e0 + 1; m < e1; ++m) s += b[l.mem[m]];
      fc[I] = s;
    }
    tm.sync();
  }
  // coarsest level: x_L = A_L^{-1} f_L (FP64 accumulation), warp per row
  T *xL = (L == 0) ? out0 : (T *)S.lev[L].y;
  {
    const T *fL = fk[L];
    const int lane = threadIdx.x & 31, wid = tm.tid >> 5, nw = tm.nthr >> 5;
    for (int i = wid; i < S.nL; i += nw) {
      const double *row = S.ainv + (size_t)i * S.nL;
      double s = 0.0;
      for (int j = lane; j < S.nL; j += 32) s += row[j] * (double)fL[j];
      s = warp_sum(s);
      if (lane == 0) xL[i] = (T)s;
    }
    tm.sync();
  }
  T *xc = xL;
  for (int k = L - 1; k >= 0; --k) {
    const BatchLevel &l = S.lev[k];
    const T *val = (const T *)l.val, *dinv = (const T *)l.dinv;
    const T *f = fk[k];
    T *fin = (k == 0) ? out0 : (T *)l.y;
    if (l.cval) {
      const T *qv = (const T *)l.qval, *wd = (const T *)l.wd, *t = (const T *)l.t;
      for (int i = tm.tid; i < l.n; i += tm.nthr)
        fin[i] = brow<T, T>(l.qrp, l.qci, qv, xc, i) + wd[i] * (f[i] + t[i]);
      tm.sync();
      xc = fin;
      continue;
    }
    T *in = cur[k];
    T *other = (in == (T *)l.x) ? (T *)l.t : (T *)l.x;
    // prolongation into `other`, then the post-smoothing sweeps, the last into fin
    T *dst0 = S.nu_post == 0 ? fin : other;
    for (int i = tm.tid; i < l.n; i += tm.nthr) dst0[i] = in[i] + xc[l.agg[i]];
    tm.sync();
    T *c = dst0, *spare = in;
    for (int sw = 0; sw < S.nu_post; ++sw) {
      T *dst = (sw == S.nu_post - 1) ? fin : spare;
      for (int i = tm.tid; i < l.n; i += tm.nthr)
        dst[i] = c[i] + omega * (dinv[i] * (f[i] - brow<T, T>(l.rp, l.ci, val, c, i)));
      tm.sync();
      spare = c;
      c = dst;
    }
    xc = fin;
  }
}

// z = M^{-1} r in FP64 at the interface; T is the V-cycle's arithmetic type.
template <typename T, int C>
__device__ void b_precond(const Team<C> &tm, const BatchSys &S, const double *r, double *z) {
  if constexpr (sizeof(T) == sizeof(double)) {
    b_vcycle<double, C>(tm, S, r, z);
  } else {
    float *f0 = (float *)S.lev[0].f, *y0 = (float *)S.lev[0].y;
    for (int i = tm.tid; i < S.n; i += tm.nthr) f0[i] = (float)r[i];
    tm.sync();
    b_vcycle<float, C>(tm, S, f0, y0);
    for (int i = tm.tid; i < S.n; i += tm.nthr) z[i] = (double)y0[i];
    tm.sync();
  }
}

// Flexible (or not) AMG-PCG of Algorithm 4 for the block's system, with the
// same stopping rule as pcg_solve: a stop on the recurrence residual whose
// true residual b - A x misses rtol replaces r by the true residual and
// restarts from x (at most BATCH_RESTARTS times), so an OK exit always has
// ||b - A x|| <= rtol ||b||.  The flexible beta is (z_{j+1}, r_{j+1} - r_j) /
// (z_j, r_j), formed as -alpha (z_{j+1}, q_j) / (z_j, r_j).
#define BATCH_RESTARTS 4
template <typename T, int C>
__global__ void __launch_bounds__(BATCH_THREADS, 1) k_batch_pcg(int nsys, const BatchJob *__restrict__ jobs,
                                                              double rtol, int max_iter, int flexible,
                                                              BatchInfo *__restrict__ info) {
  __shared__ double sh[33];
  const int sidx = blockIdx.x / C;  // the whole team leaves together
  if (sidx >= nsys) return;
  const Team<C> tm;
  const BatchSys &S = *jobs[sidx].sys;
  const double *b = jobs[sidx].b;
  double *x = jobs[sidx].x;
  const int n = S.n;
  double *r = S.r, *z = S.z, *p = S.p, *q = S.q;
  // ||b||, and r = b - A x with its norm
  auto residual = [&](double *bb_out) {
    double bb = 0.0, rr = 0.0;
    for (int i = tm.tid; i < n; i += tm.nthr) {
      const double ri = b[i] - brow<double, double>(S.rp0, S.ci0, S.val0, x, i);
      r[i] = ri;
      bb += b[i] * b[i];
      rr += ri * ri;
    }
    bb = tm.sum(bb, sh);
    rr = tm.sum(rr, sh);
    if (bb_out) *bb_out = bb;
    return rr;
  };
  double bb = 0.0;
  double rr = residual(&bb);
  const double bnorm = sqrt(bb);
  double rel = bnorm > 0.0 ? sqrt(rr) / bnorm : 0.0;
  int it = 0, status = AMG_ERR_NOT_CONVERGED;
  if (!isfinite(bb) || !isfinite(rr)) {
    status = AMG_ERR_INVALID_ARG;
  } else if (bnorm == 0.0) {
    for (int i = tm.tid; i < n; i += tm.nthr) x[i] = 0.0;
    status = AMG_OK;
  } else if (rel <= rtol) {
    status = AMG_OK;
  } else if (max_iter > 0) {
    for (int restart = 0;; ++restart) {
      tm.sync();
      b_precond<T, C>(tm, S, r, z);
      double rz = 0.0;
      for (int i = tm.tid; i < n; i += tm.nthr) { p[i] = z[i]; rz += r[i] * z[i]; }
      rz = tm.sum(rz, sh);
      status = AMG_ERR_NOT_CONVERGED;
      while (it < max_iter) {
        tm.sync();
        double pq = 0.0;
        for (int i = tm.tid; i < n; i += tm.nthr) {
          const double qi = brow<double, double>(S.rp0, S.ci0, S.val0, p, i);
          q[i] = qi;
          pq += p[i] * qi;
        }
        pq = tm.sum(pq, sh);
        if (pq == 0.0 || !isfinite(pq) || !isfinite(rz)) { status = AMG_ERR_BREAKDOWN; break; }
        const double alpha = rz / pq;
        double r2 = 0.0;
        for (int i = tm.tid; i < n; i += tm.nthr) {
          x[i] = x[i] + alpha * p[i];
          const double ri = r[i] - alpha * q[i];
          r[i] = ri;
          r2 += ri * ri;
        }
        r2 = tm.sum(r2, sh);
        ++it;
        rel = sqrt(r2) / bnorm;
        if (rel <= rtol) { status = AMG_OK; break; }
        if (!isfinite(rel)) { status = AMG_ERR_BREAKDOWN; break; }
        if (it == max_iter) break;
        tm.sync();
        b_precond<T, C>(tm, S, r, z);
        double rzn = 0.0, zq = 0.0;
        for (int i = tm.tid; i < n; i += tm.nthr) {
          rzn += r[i] * z[i];
          if (flexible) zq += z[i] * q[i];
        }
        rzn = tm.sum(rzn, sh);
        if (flexible) zq = tm.sum(zq, sh);
        const double beta = (flexible ? -alpha * zq : rzn) / rz;
        if (!isfinite(beta)) { status = AMG_ERR_BREAKDOWN; break; }
        rz = rzn;
        tm.sync();
        for (int i = tm.tid; i < n; i += tm.nthr) p[i] = z[i] + beta * p[i];
      }
      if (status != AMG_OK || restart >= BATCH_RESTARTS || it >= max_iter) break;
      // true residual: accept, or restart from x with r = b - A x
      tm.sync();
      rr = residual(nullptr);
      rel = sqrt(rr) / bnorm;
      if (rel <= rtol) break;
      if (!isfinite(rel)) { status = AMG_ERR_BREAKDOWN; break; }
      status = AMG_ERR_NOT_CONVERGED;
    }
  }
  tm.sync();
  // true relative residual from x
  double tr = 0.0;
  for (int i = tm.tid; i < n; i += tm.nthr) {
    double ri = b[i] - brow<double, double>(S.rp0, S.ci0, S.val0, x, i);
    tr += ri * ri;
  }
  tr = tm.sum(tr, sh);
  if (tm.tid == 0) {
    info[sidx].iterations = it;
    info[sidx].status = status;
    info[sidx].rel = rel;
    info[sidx].rel_true = bnorm > 0.0 ? sqrt(tr) / bnorm : 0.0;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

// Builds (once) the device descriptor of a hierarchy for batched solves.
amg_status batch_descriptor(amg_hierarchy *h, cudaStream_t s, const BatchSys **out) {
  if (h->batch_desc && !h->batch_desc_stale) { *out = (const BatchSys *)h->batch_desc; return AMG_OK; }
  if (!h->dense || !h->ainv || h->lev[h->L].n > BATCH_MAX_COARSE) return AMG_ERR_UNSUPPORTED;
  if (h->prm.precision == AMG_FP16_STORAGE) return AMG_ERR_UNSUPPORTED;
  if (h->prm.cycle != AMG_CYCLE_V) return AMG_ERR_UNSUPPORTED;
  const bool f32 = h->prm.precision == AMG_FP32;
  BatchSys d = {};
  d.L = h->L;
  d.n = h->lev[0].n;
  d.nL = h->lev[h->L].n;
  d.omega = h->prm.omega;
  d.nu_pre = h->prm.nu_pre;
  d.nu_post = h->prm.nu_post;
  for (int k = 0; k <= h->L; ++k) {
    Level &l = h->lev[k];
    BatchLevel &b = d.lev[k];
    b.n = l.n;
    b.nc = k < h->L ? h->lev[k + 1].n : 0;
    b.rp = l.rp;
    b.ci = l.ci;
    b.val = f32 ? (const void *)l.val32 : (const void *)l.val;
    b.dinv = f32 ? (const void *)l.dinv32 : (const void *)l.dinv;
    b.agg = l.agg;
    b.mrp = l.mrp;
    b.mem = l.mem;
    b.f = f32 ? (void *)l.f32 : (void *)l.f;
    b.x = f32 ? (void *)l.x32 : (void *)l.x;
    b.t = f32 ? (void *)l.t32 : (void *)l.t;
    b.y = f32 ? (void *)l.y32 : (void *)l.y;
    const bool op = k < h->L && l.op_avail && l.op_on;
    b.cval = op ? (f32 ? (const void *)l.cval32 : (const void *)l.cval) : nullptr;
    b.qval = op ? (f32 ? (const void *)l.qval32 : (const void *)l.qval) : nullptr;
    b.wd = op ? (f32 ? (const void *)l.wd32 : (const void *)l.wd) : nullptr;
    b.qrp = op ? l.qrp : nullptr;
    b.qci = op ? l.qci : nullptr;
  }
  d.ainv = h->ainv;
  d.rp0 = h->lev[0].rp;
  d.ci0 = h->lev[0].ci;
  d.val0 = h->lev[0].val;
  d.r = h->kr;
  d.z = h->kz;
  d.p = h->kp;
  d.q = h->kq;
  d.rold = h->krold;
  void *dev = h->batch_desc;  // rebuilt in place when the levels' forms changed
  if (!dev) AMG_TRY(hier_alloc(h, &dev, sizeof(BatchSys)));
  AMG_CUDA(cudaMemcpyAsync(dev, &d, sizeof(BatchSys), cudaMemcpyHostToDevice, s));
  AMG_CUDA(cudaStreamSynchronize(s));
  h->batch_desc = dev;
  h->batch_desc_stale = 0;
  *out = (const BatchSys *)dev;
  return AMG_OK;
}

// nsys systems of one team size: nsys * team blocks, clusters of `team`.
template <typename T>
cudaError_t launch_batch(int team, int nsys, const BatchJob *jobs, double rtol, int max_iter, int flexible,
                         BatchInfo *info, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nsys * team));
  cfg.blockDim = dim3(BATCH_THREADS);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)team;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = team > 1 ? 1 : 0;
  switch (team) {
    case 1: return cudaLaunchKernelEx(&cfg, k_batch_pcg<T, 1>, nsys, jobs, rtol, max_iter, flexible, info);
    case 2: return cudaLaunchKernelEx(&cfg, k_batch_pcg<T, 2>, nsys, jobs, rtol, max_iter, flexible, info);
    case 4: return cudaLaunchKernelEx(&cfg, k_batch_pcg<T, 4>, nsys, jobs, rtol, max_iter, flexible, info);
    default: return cudaLaunchKernelEx(&cfg, k_batch_pcg<T, 8>, nsys, jobs, rtol, max_iter, flexible, info);
  }
}

}  // namespace

extern "C" amg_status amg_batch_pcg(int nsys, amg_hierarchy *const *hs, const double *const *d_b,
                                    double *const *d_x, double rtol, int max_iter, int flexible,
                                    amg_stream_t stream, amg_solve_info *infos) {
  clear_stale_cuda_error();
  if (nsys <= 0 || !hs || !d_b || !d_x || !(rtol >= 0.0) || max_iter < 0) return AMG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int prec = -1;
  std::vector<BatchJob> jobs(nsys);
  for (int i = 0; i < nsys; ++i) {
    if (!hs[i] || !d_b[i] || !d_x[i]) return AMG_ERR_INVALID_ARG;
    if (prec < 0) prec = hs[i]->prm.precision;
    if (hs[i]->prm.precision != prec) return AMG_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return AMG_ERR_INVALID_ARG;  // a hierarchy's work vectors serve one solve
    AMG_TRY(batch_descriptor(hs[i], s, &jobs[i].sys));
    hs[i]->last_stream = s;
    jobs[i].b = d_b[i];
    jobs[i].x = d_x[i];
  }
  BatchJob *d_jobs = nullptr;
  BatchInfo *d_info = nullptr;
  AMG_TRY(pool_alloc((void **)&d_jobs, sizeof(BatchJob) * nsys, s));
  if (pool_alloc((void **)&d_info, sizeof(BatchInfo) * nsys, s) != AMG_OK) {
    pool_free(d_jobs, s);
    return AMG_ERR_OOM;
  }
  std::vector<BatchInfo> hinfo(nsys);
  // one launch per team size, the systems of each size contiguous
  std::vector<int> order(nsys);
  for (int i = 0; i < nsys; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return batch_team(hs[a]->lev[0].n) < batch_team(hs[b]->lev[0].n); });
  std::vector<BatchJob> sorted(nsys);
  for (int i = 0; i < nsys; ++i) sorted[i] = jobs[order[i]];
  cudaError_t e = cudaMemcpyAsync(d_jobs, sorted.data(), sizeof(BatchJob) * nsys, cudaMemcpyHostToDevice, s);
  for (int g0 = 0; g0 < nsys && e == cudaSuccess;) {
    const int team = batch_team(hs[order[g0]]->lev[0].n);
    int g1 = g0;
    while (g1 < nsys && batch_team(hs[order[g1]]->lev[0].n) == team) ++g1;
    e = prec == AMG_FP32 ? launch_batch<float>(team, g1 - g0, d_jobs + g0, rtol, max_iter, flexible, d_info + g0, s)
                         : launch_batch<double>(team, g1 - g0, d_jobs + g0, rtol, max_iter, flexible, d_info + g0, s);
    count_launch();
    g0 = g1;
  }
  std::vector<BatchInfo> sinfo(nsys);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sinfo.data(), d_info, sizeof(BatchInfo) * nsys, cudaMemcpyDeviceToHost, s);
  pool_free(d_jobs, s);
  pool_free(d_info, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return amg_cuda_status(e);
  for (int i = 0; i < nsys; ++i) hinfo[order[i]] = sinfo[i];
  amg_status worst = AMG_OK;
  for (int i = 0; i < nsys; ++i) {
    if (infos) {
      infos[i].iterations = hinfo[i].iterations;
      infos[i].rel_res_recurrence = hinfo[i].rel;
      infos[i].rel_res_true = hinfo[i].rel_true;
      infos[i].status = (amg_status)hinfo[i].status;
    }
    if (hinfo[i].status != AMG_OK && worst == AMG_OK) worst = (amg_status)hinfo[i].status;
  }
  return worst;
}
