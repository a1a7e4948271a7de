// cluster_cg.cu -- coarsest solve of small stalled hierarchies on one thread
// block cluster.
//
// The coarsest-level CG (Jacobi-PCG to a relative residual of 1e-12, the CG
// coarse solver compared in Sec. 4.2) in the same pipelined arrangement as the
// grid-wide kernel k_coarse_cg (Ghysels and Vanroose 2014: one synchronisation
// per iteration publishes the preconditioned vector m = D^-1 w and the block
// partial sums together), but on the CTAs of one cluster instead of a
// cooperative grid.  Each CTA keeps its rows' CG vectors in shared memory;
// the matrix product gathers m from the owning CTA's shared memory through the
// cluster's distributed shared memory, the inner products are summed from the
// CTAs' partials the same way, and the synchronisation is the hardware cluster
// barrier rather than an atomic counter in global memory.  A coarsest level of
// up to about two thousand rows is bound by synchronisation and latency, not
// by FP64 work, and 16 SMs with the cluster barrier finish an iteration
// 15-20% sooner than the grid-wide kernel (5.2 against 6.6 us at 1728 rows);
// from about four thousand rows the FP64 work of 16 SMs makes it slower.
// 128 threads per CTA (one row per thread up to 2048 rows): block barriers
// over four warps cost less than over sixteen, and they dominate the stalls.
//
// Rows are split into C contiguous ranges of `rows_per` rows (the last ones
// may be short or empty); the owner of column c is c / rows_per.  m and the
// partials are double buffered by iteration parity: a CTA writes the buffer
// of iteration it+1 only after the barrier of iteration it, which every CTA
// reaches after its last read of that buffer (iteration it-1's product).
// All CTAs compute the scalars from the same partials in the same order, so
// they take the same decisions and leave the loop together; a last barrier
// keeps every CTA's shared memory alive until the others' final reads.
#include <cooperative_groups.h>

#include "common.cuh"

namespace cgr = cooperative_groups;

#define CCG_THREADS 128
#define CCG_RTOL 1e-12
#define CCG_MAXIT 1000
#define CCG_GATHER 8      // neighbours gathered per round by one thread
#define CCG_VECS 12       // r u w z q s p x d n, m[2]

namespace {

// Owner CTA of column c and its index there (c < 2^24, rows_per >= 1).
__device__ __forceinline__ int ccg_owner(int c, int rows_per, float inv_rows) {
  int o = (int)((float)c * inv_rows);
  if (o * rows_per > c) --o;
  else if ((o + 1) * rows_per <= c) ++o;
  return o;
}

template <typename T>
__global__ void __launch_bounds__(CCG_THREADS)
    k_coarse_cg_cluster(int n, int rows_per, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                        const double *__restrict__ val, const double *__restrict__ dinv, const T *__restrict__ f,
                        T *__restrict__ xout, int *iters, unsigned long long *iters_total, const KState *st) {
  if (is_done(st)) return;  // the same for every CTA: no barrier has been reached yet
  cgr::cluster_group cluster = cgr::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  extern __shared__ __align__(16) double ccg_sm[];
  __shared__ double red[3][CCG_THREADS];
  __shared__ double part[2][4];  // block partials (r,u), (w,u), (r,r) by parity; read by every CTA
  __shared__ double tot_sh[3], sc[3], rcp_sh[2];
  const int r0 = rank * rows_per;
  const int nr = max(0, min(rows_per, n - r0));
  const float inv_rows = 1.0f / (float)rows_per;
  double *vr = ccg_sm, *vu = vr + rows_per, *vw = vu + rows_per, *vz = vw + rows_per;
  double *vq = vz + rows_per, *vs = vq + rows_per, *vp = vs + rows_per, *vx = vp + rows_per;
  double *vd = vx + rows_per, *vn = vd + rows_per;
  double *const m0 = vn + rows_per, *const m1 = vn + 2 * rows_per;  // m by iteration parity
  auto mbuf = [&](int p) { return p ? m1 : m0; };
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // y = A v for the CTA's rows, v distributed over the cluster (buffer vb of
  // every CTA); CCG_GATHER independent gathers in flight per thread
  auto spmv = [&](double *vb, double *vy) {
    for (int t = tid; t < nr; t += CCG_THREADS) {
      const int i = r0 + t;
      const int b = rp[i], e = rp[i + 1];
      double y = 0.0;
      for (int e0 = b; e0 < e; e0 += CCG_GATHER) {
        double a[CCG_GATHER], xv[CCG_GATHER];
#pragma unroll
        for (int k = 0; k < CCG_GATHER; ++k) {
          const int ee = e0 + k;
          const bool in = ee < e;
          const int c = in ? __ldg(&ci[ee]) : i;
          a[k] = in ? __ldg(&val[ee]) : 0.0;
          const int o = ccg_owner(c, rows_per, inv_rows);
          const double *src = o == rank ? vb : cluster.map_shared_rank(vb, o);
          xv[k] = src[c - o * rows_per];
        }
#pragma unroll
        for (int k = 0; k < CCG_GATHER; ++k) y = __fma_rn(a[k], xv[k], y);
      }
      vy[t] = y;
    }
  };
  // block partials of three inner products into part[slot] (whole-warp
  // halving in shared memory: predicated-off FP64 lanes cost as much as
  // active ones)
  auto block_partials = [&](double (&v)[3], int slot) {
    red[0][tid] = v[0];
    red[1][tid] = v[1];
    red[2][tid] = v[2];
    __syncthreads();
    for (int h = CCG_THREADS >> 1; h >= 32; h >>= 1) {
      if (tid < h) {
        red[0][tid] += red[0][tid + h];
        red[1][tid] += red[1][tid + h];
        red[2][tid] += red[2][tid + h];
      }
      __syncthreads();
    }
    if (warp < 3) {
      const double s = warp_sum(red[warp][lane]);
      if (lane == 0) part[slot][warp] = s;
    }
  };

  // initial phase: r = f, u = D^-1 f (published), the other vectors zero
  for (int t = tid; t < nr; t += CCG_THREADS) {
    const int i = r0 + t;
    const double fi = (double)f[i];
    const double di = __ldg(&dinv[i]);
    const double ui = __dmul_rn(fi, di);
    vd[t] = di;
    vr[t] = fi;
    vu[t] = ui;
    m1[t] = ui;
    vz[t] = 0.0;
    vq[t] = 0.0;
    vs[t] = 0.0;
    vp[t] = 0.0;
    vx[t] = 0.0;
  }
  cluster.sync();
  spmv(m1, vw);  // w = A u
  double acc[3] = {0.0, 0.0, 0.0};
  for (int t = tid; t < nr; t += CCG_THREADS) {
    const double ri = vr[t], ui = vu[t], wi = vw[t];
    m0[t] = __dmul_rn(wi, vd[t]);
    acc[0] = __fma_rn(ri, ui, acc[0]);
    acc[1] = __fma_rn(wi, ui, acc[1]);
    acc[2] = __fma_rn(ri, ri, acc[2]);
  }
  double thresh = 0.0;
  int it = 0;
  for (it = 0;; ++it) {
    const int par = it & 1;
    block_partials(acc, par);
    cluster.sync();  // m of this iteration and the partials are visible cluster-wide
    spmv(mbuf(par), vn);  // n = A m
    if (warp == 0) {
      // totals: lane q reads CTA q's partials (C <= 32), then a fixed shuffle
      // tree -- the same sums, in the same order, on every CTA
      double g = 0.0, d = 0.0, rr = 0.0;
      if (lane < C) {
        const double *pq = cluster.map_shared_rank(&part[par][0], lane);
        g = pq[0];
        d = pq[1];
        rr = pq[2];
      }
      g = warp_sum(g);
      d = warp_sum(d);
      rr = warp_sum(rr);
      if (lane == 0) {
      tot_sh[0] = g;
      tot_sh[1] = d;
      tot_sh[2] = rr;
      if (it == 0) thresh = (CCG_RTOL * sqrt(rr)) * (CCG_RTOL * sqrt(rr));
      bool stop = rr <= thresh || it >= CCG_MAXIT;
      double a = 0.0, bt = 0.0;
      if (!stop) {
        if (it == 0) {
          a = g / d;
        } else {
          bt = g * rcp_sh[0];
          a = g / (d - g * g * rcp_sh[1]);
        }
        stop = !isfinite(a);
      }
      sc[0] = a;
      sc[1] = bt;
      sc[2] = stop ? 1.0 : 0.0;
      }
    }
    __syncthreads();
    if (sc[2] != 0.0) break;
    const double alpha = sc[0], beta = sc[1];
    // the next iteration's 1/gamma and 1/(gamma alpha), off the critical path
    if (tid == 32) rcp_sh[0] = 1.0 / tot_sh[0];
    if (tid == 64) rcp_sh[1] = 1.0 / (tot_sh[0] * alpha);
    const double *vm = mbuf(par);
    double *mnext = mbuf(par ^ 1);
    acc[0] = acc[1] = acc[2] = 0.0;
    for (int t = tid; t < nr; t += CCG_THREADS) {
      const double zi = __fma_rn(beta, vz[t], vn[t]);
      const double qi = __fma_rn(beta, vq[t], vm[t]);
      const double si = __fma_rn(beta, vs[t], vw[t]);
      const double pi = __fma_rn(beta, vp[t], vu[t]);
      vx[t] = __fma_rn(alpha, pi, vx[t]);
      const double ri = __fma_rn(-alpha, si, vr[t]);
      const double ui = __fma_rn(-alpha, qi, vu[t]);
      const double wi = __fma_rn(-alpha, zi, vw[t]);
      vz[t] = zi;
      vq[t] = qi;
      vs[t] = si;
      vp[t] = pi;
      vr[t] = ri;
      vu[t] = ui;
      vw[t] = wi;
      mnext[t] = __dmul_rn(wi, vd[t]);
      acc[0] = __fma_rn(ri, ui, acc[0]);
      acc[1] = __fma_rn(wi, ui, acc[1]);
      acc[2] = __fma_rn(ri, ri, acc[2]);
    }
  }
  for (int t = tid; t < nr; t += CCG_THREADS) xout[r0 + t] = (T)vx[t];
  if (rank == 0 && tid == 0) {
    *iters = it;
    atomicAdd(iters_total, (unsigned long long)it);
  }
  cluster.sync();  // no CTA leaves while another may still read its shared memory
}

template <typename T>
cudaError_t ccg_launch_t(const ClusterCG &cc, int n, const int32_t *rp, const int32_t *ci, const double *val,
                         const double *dinv, const T *f, T *x, int *iters, unsigned long long *iters_total,
                         const KState *st, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cc.size);
  cfg.blockDim = dim3(CCG_THREADS);
  cfg.dynamicSmemBytes = cc.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cc.size;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_coarse_cg_cluster<T>, n, cc.rows_per, rp, ci, val, dinv, f, x, iters,
                            iters_total, st);
}

// The kernel's attributes are process-wide, so they are set to fixed values
// (the largest shared memory any configuration uses), never to one
// hierarchy's size: a setup on another thread must not lower the limit under
// a launch that needs more.
#define CCG_SMEM_CAP (200 * 1024)

template <typename T>
cudaError_t ccg_prepare_kernel() {
  cudaError_t e = cudaFuncSetAttribute(k_coarse_cg_cluster<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_coarse_cg_cluster<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, CCG_SMEM_CAP);
  return e;
}

template <typename T>
int ccg_max_clusters(int size, size_t smem) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(size);
  cfg.blockDim = dim3(CCG_THREADS);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = size;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int num = 0;
  if (cudaOccupancyMaxActiveClusters(&num, k_coarse_cg_cluster<T>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return num;
}

}  // namespace

// Chooses the cluster solver for an n-row coarsest level: the largest cluster
// size (16, non-portable, else 8) that the device can schedule with the
// shared memory of ceil(n / size) rows, if n <= CCG_MAX_N.  cc->size = 0
// leaves the level to the grid-wide kernel.
amg_status cluster_cg_config(int n, ClusterCG *cc) {
  cc->size = 0;
  if (n < 1 || n > CCG_MAX_N) return AMG_OK;
  for (int size : {16, 8}) {
    const int rows_per = cdiv(n, size);
    const size_t smem = sizeof(double) * (size_t)CCG_VECS * rows_per;
    if (smem > CCG_SMEM_CAP) continue;
    if (ccg_prepare_kernel<double>() != cudaSuccess || ccg_prepare_kernel<float>() != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (ccg_max_clusters<double>(size, smem) < 1 || ccg_max_clusters<float>(size, smem) < 1) continue;
    cc->size = size;
    cc->rows_per = rows_per;
    cc->smem = smem;
    return AMG_OK;
  }
  return AMG_OK;
}

template <typename T>
amg_status cluster_cg_launch(const ClusterCG &cc, int n, const int32_t *rp, const int32_t *ci, const double *val,
                             const double *dinv, const T *f, T *x, int *iters, unsigned long long *iters_total,
                             const KState *st, cudaStream_t s) {
  // the caller's LaunchScope counts the launch
  if (cc.size < 1 || (long long)cc.size * cc.rows_per < n) return AMG_ERR_INVALID_ARG;
  return amg_cuda_status(ccg_launch_t<T>(cc, n, rp, ci, val, dinv, f, x, iters, iters_total, st, s));
}
template amg_status cluster_cg_launch<double>(const ClusterCG &, int, const int32_t *, const int32_t *,
                                              const double *, const double *, const double *, double *, int *,
                                              unsigned long long *, const KState *, cudaStream_t);
template amg_status cluster_cg_launch<float>(const ClusterCG &, int, const int32_t *, const int32_t *,
                                             const double *, const double *, const float *, float *, int *,
                                             unsigned long long *, const KState *, cudaStream_t);
