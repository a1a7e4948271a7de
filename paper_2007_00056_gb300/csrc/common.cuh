// common.cuh -- internal declarations of the GB300 aggregation-AMG library.
//
// Device data layout (all in HBM, owned by the hierarchy):
//   level k:  rp[n+1], ci[nnz] (int32), val[nnz] (FP64) + val32[nnz] (FP32
//             copy for the mixed-precision V-cycle) + val16/dscale (FP16
//             storage of D^-1/2 A D^-1/2), dinv[n] = 1/a_ii (FP64 and FP32);
//             agg[n] fine->coarse map and the member lists of every coarse
//             aggregate (mrp[n_c+1], mem[n]; members ascending) for k < L;
//             per-level V-cycle vectors f, x, t.
//   coarsest: dense inverse A_L^{-1} (row-major FP64) or the coarse-CG work
//             vectors.
//   Krylov:   level-0 FP64 work vectors and a device-resident scalar block
//             (KState) so an iteration runs without host round trips.
// After amg_set_residency, the matrix arrays (column indices and values) of
// the chosen levels live in pinned host memory instead (residency.cu).
// Every CSR array is padded by AMG_PAD elements so that vector loads of a
// tile never leave the allocation.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "amg.h"

#define AMG_MAX_LEVELS 32
#define AMG_MAX_PASSES 8
#define AMG_PAD 64
#define AMG_THREADS 256
#define AMG_MAX_BLOCKS 2432  // 152 SMs x 16 resident 256-thread blocks (upper bound of any grid)

// Device error flags (bit set, read back by the host at the next sync point).
#define AMG_EFLAG_ZERO_DIAG 1u
#define AMG_EFLAG_NONSYM 2u
#define AMG_EFLAG_TIMEOUT 4u
#define AMG_EFLAG_BAD_CSR 8u
#define AMG_EFLAG_BREAKDOWN 16u
#define AMG_EFLAG_NONFINITE 32u

// Krylov state held on the device; kernels read the scalars they need and the
// reduction finalisers write the next ones.  `done` makes every later kernel
// of the solve a no-op, so the host can enqueue several iterations at once.
struct KState {
  double rz, pq, alpha, beta, omega, rho, bnorm, rel, rtol, srel, rel_true;
  int it, max_iter, done, status, flexible, half;
  int xpend;  // PCG: the last iteration's x += alpha p is still to be applied
};

struct Level {
  int n = 0;
  int64_t nnz = 0;
  int32_t *rp = nullptr, *ci = nullptr;
  double *val = nullptr, *dinv = nullptr;
  float *val32 = nullptr, *dinv32 = nullptr;
  __half *val16 = nullptr;   // values of D^-1/2 A D^-1/2 (FP16 storage mode, levels < L)
  float *sig = nullptr;      // sqrt(a_ii)        (FP16 storage mode)
  float *isig = nullptr;     // 1 / sqrt(a_ii)    (FP16 storage mode)
  int32_t *agg = nullptr;    // n, into level k+1
  int32_t *mrp = nullptr;    // n_{k+1}+1
  int32_t *mem = nullptr;    // n
  int32_t *perm = nullptr;   // row processing order grouped by length class (levels >= 1)
  double *f = nullptr, *x = nullptr, *t = nullptr, *y = nullptr;
  float *f32 = nullptr, *x32 = nullptr, *t32 = nullptr, *y32 = nullptr;
  int rounds[AMG_MAX_PASSES] = {0};
  int tpr = 1;               // threads per row of this level's row kernels
  int st_cap = 0;            // TMA-staged row kernels: entries per stage buffer (0: not offered)
  int st_grid = 0;           // blocks of the persistent staged kernels
  int fuse_pre = 1;          // first presmoothing sweep fused into the residual kernel
  int fuse_post = 0;         // prolongation fused into the first postsmoothing sweep
  // Residual-operator form of a cycle visit from the zero guess with one pre-
  // and one post-smoothing sweep (levels < L; FP64 values, FP32 copies in the
  // FP32 mode).  With x = omega D^-1 f the presmoothed iterate:
  //   t = f - A x = C f,                     C = I - omega A D^-1 (pattern of A)
  //   y = x + P x_c + omega D^-1 (t - A P x_c) = Q x_c + wd (f + t),
  //                                          Q = P - omega D^-1 A P, wd = omega D^-1
  // so the visit reads one matrix of A's size and one of A P's size, and
  // never stores x.
  double *cval = nullptr, *qval = nullptr, *wd = nullptr;
  float *cval32 = nullptr, *qval32 = nullptr, *wd32 = nullptr;
  int32_t *qrp = nullptr, *qci = nullptr;  // CSR pattern of A P (n x n_{k+1}), columns ascending
  int64_t qnnz = 0;
  int op_avail = 0;          // C, Q and wd exist for this level
  int op_on = 0;             // zero-guess visits use them
  int host = 0;              // its matrix arrays are in pinned host memory (residency.cu)
  int st_cap_dev = 0;        // st_cap while the level was in device memory
};

// Kernel kinds of the per-kernel profiler (id = kind * AMG_MAX_LEVELS + level).
enum ProfKind {
  PK_JACOBI0 = 0, PK_JACOBI, PK_RESIDUAL, PK_RESTRICT, PK_PROLONG_JACOBI, PK_PROLONG, PK_COARSE_DENSE,
  PK_COARSE_CG, PK_CAST, PK_KRYLOV_SPMV, PK_KRYLOV_VEC, PK_OP_RESIDUAL, PK_OP_POST, PK_COUNT
};
#define AMG_PROF_IDS (PK_COUNT * AMG_MAX_LEVELS)

// Optional CUDA-event timing of every solve-phase launch (off by default;
// while on, iterations run as direct launches instead of graph replays).
struct Profiler {
  bool on = false;
  struct Rec { int id; double bytes; cudaEvent_t a, b; };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  double ms[AMG_PROF_IDS] = {0};
  double bytes[AMG_PROF_IDS] = {0};
  long long launches[AMG_PROF_IDS] = {0};
};

// Work memory of the persistent coarse CG: the published halo vector (double
// buffered by iteration parity), the row state when it does not fit in shared
// memory (CG_STATE vectors of n + AMG_PAD, by position), reduction partials,
// barrier counter and iteration counters.
#define CG_STATE 10                 // r, u, w, m, n, z, q, s, p, x
// Coarsest CG on one thread block cluster (cluster_cg.cu): used for coarsest
// levels of at most CCG_MAX_N rows when the device schedules the cluster;
// size = 0 leaves the level to the grid-wide kernel.
#define CCG_MAX_N 2048
struct ClusterCG {
  int size = 0;       // CTAs in the cluster (16 or 8)
  int rows_per = 0;   // rows per CTA
  size_t smem = 0;    // dynamic shared memory per CTA
};

struct CoarseCG {
  int n = 0, grid = 0, threads = 0;
  size_t smem = 0;           // dynamic shared memory per block (matrix slice staging)
  double *halo[2] = {nullptr, nullptr};
  double *state = nullptr;
  double *part = nullptr;    // CG_PART_DOUBLES: 2 slots x 3 values x AMG_MAX_BLOCKS
  int *ord = nullptr;        // n: rows of each block's range sorted by length (coarse_cg_prepare)
  int *meta = nullptr;       // 5 x grid: row range and length-group bounds per block
  unsigned *bar = nullptr;   // [0] monotonic arrival counter
  int *iters = nullptr;
  unsigned long long *iters_total = nullptr;  // sum of CG iterations over launches
  ClusterCG cl;              // cluster form for small levels (cl.size = 0: not used)
};

struct amg_hierarchy {
  amg_params prm{};
  int device = 0;
  int num_sms = 152;
  int L = 0;                 // index of the coarsest level
  Level lev[AMG_MAX_LEVELS];
  int dense = 0;
  double *ainv = nullptr;    // n_L x n_L, row-major FP64 inverse (null when ainv32 is used)
  float *ainv32 = nullptr;   // n_L x n_L, row-major FP32 inverse, refined in FP64 per solve
  double *dense_r = nullptr; // 2 x n_L: refinement residual and FP64 working solution
  int dense_refine = 0;      // refinement steps per coarse solve with ainv32
  CoarseCG cg;
  // Krylov work vectors (level 0, FP64)
  double *kb = nullptr, *kx = nullptr, *kr = nullptr, *kz = nullptr, *kp = nullptr, *kq = nullptr;
  double *krold = nullptr, *ks = nullptr, *kt = nullptr, *krb = nullptr, *kph = nullptr, *ksh = nullptr;
  double *part = nullptr;    // reduction partials, 8 x AMG_MAX_BLOCKS
  unsigned *counter = nullptr;  // last-block counters, 8 slots
  KState *st = nullptr;      // device
  KState *st_host = nullptr; // pinned host mirror
  unsigned *eflags = nullptr;   // device error bits
  unsigned *eflags_host = nullptr;
  std::vector<std::pair<void *, size_t>> allocs;       // device memory owned, with sizes
  std::vector<std::pair<void *, size_t>> host_allocs;  // pinned host memory owned (moved level arrays)
  int residency = 0;         // amg_residency
  int res_first = 0;         // first level whose matrix arrays are in host memory
  struct Stager *stg = nullptr;  // two-slot staging of host-resident levels (AMG_HOST_STAGED)
  cudaStream_t stream = nullptr;       // stream of amg_setup (stream-ordered allocations)
  cudaStream_t last_stream = nullptr;  // stream of the latest call that used the hierarchy
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t g_vcycle = nullptr, g_pcg = nullptr, g_bicg = nullptr, g_amg = nullptr;
  long long g_pcg_nodes = 0, g_bicg_nodes = 0, g_amg_nodes = 0;
  int graphs_ok = 1;
  int solves = 0;            // Krylov solves run on this hierarchy (graphs from the second one)
  Profiler prof;
  void *batch_desc = nullptr;  // device descriptor for batched solves (built on first use)
  int batch_desc_stale = 0;    // the levels' kernel forms changed since it was built
};

// Kernel launches issued by this library since it was loaded (graph replays
// count every kernel node they run).
extern unsigned long long g_amg_launches;
static inline void count_launch(long long k = 1) { __atomic_add_fetch(&g_amg_launches, (unsigned long long)k, __ATOMIC_RELAXED); }

void prof_begin(amg_hierarchy *h, cudaStream_t s, int id, double bytes);
void prof_end(amg_hierarchy *h, cudaStream_t s);
amg_status prof_flush(amg_hierarchy *h);
// Brackets one launch: counts it and, when profiling is on, times it.
struct LaunchScope {
  amg_hierarchy *h;
  cudaStream_t s;
  bool on;
  LaunchScope(amg_hierarchy *h_, cudaStream_t s_, int kind, int level, double bytes)
      : h(h_), s(s_), on(h_ != nullptr && h_->prof.on) {
    count_launch();
    if (on) prof_begin(h, s, kind * AMG_MAX_LEVELS + level, bytes);
  }
  ~LaunchScope() {
    if (on) prof_end(h, s);
  }
};

// ---------------------------------------------------------------------------
// Host helpers (defined in api.cu)
// ---------------------------------------------------------------------------
amg_status amg_cuda_status(cudaError_t e);
// Clears the calling thread's last CUDA error at a public entry point, so that
// the checks after this call's own launches report this call's errors and not
// an error some other code of the thread left behind.
static inline void clear_stale_cuda_error() { (void)cudaGetLastError(); }
// The same, recording the library source location of the failing call for
// amg_last_cuda_error.
amg_status amg_cuda_status_at(cudaError_t e, const char *file, int line);
amg_status hier_alloc(amg_hierarchy *h, void **p, size_t bytes);
// Records device memory allocated from the pool as owned by the hierarchy.
static inline void hier_adopt(amg_hierarchy *h, void *p, size_t bytes) { h->allocs.push_back({p, bytes}); }
// Stream-ordered allocation from the library's own device memory pool (freed
// memory stays in the pool for the next setup; no implicit device sync).
amg_status pool_alloc(void **p, size_t bytes, cudaStream_t s);
void pool_free(void *p, cudaStream_t s);
// Returns the pool's unused blocks to the device.
void pool_trim();
// Recycled pinned host buffers of 256 bytes (status and counter read-backs).
void *pinned_small_alloc();
void pinned_small_free(void *p);
#define AMG_TRY(x)                              \
  do {                                          \
    amg_status _s = (x);                        \
    if (_s != AMG_OK) return _s;                \
  } while (0)
#define AMG_CUDA(x)                             \
  do {                                          \
    cudaError_t _e = (x);                       \
    if (_e != cudaSuccess) return amg_cuda_status_at(_e, __FILE__, __LINE__); \
  } while (0)

// Host-resident levels (residency.cu).  A cycle visit of level k reads one
// matrix: A (explicit sweeps), C (residual-operator form, descending) or Q
// (residual-operator form, ascending).  With AMG_HOST_STAGED, stage_acquire
// returns the level with that matrix's host-resident arrays replaced by a
// device staging buffer (the stream waits for the copy), and stage_release,
// called once the visit's kernels are enqueued, frees the buffer for the
// copy of a later visit and starts the copy of the predicted next one.
enum StageSet { SET_A = 0, SET_C = 1, SET_Q = 2, SET_NONE = 3 };
static inline bool stage_on(const amg_hierarchy *h, int k) { return h->stg != nullptr && h->lev[k].host; }
Level stage_acquire(amg_hierarchy *h, int k, int set, cudaStream_t s);
void stage_release(amg_hierarchy *h, int k, bool descending, cudaStream_t s);
void residency_release(amg_hierarchy *h);  // frees host memory and the stager (amg_destroy)

static inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }
static inline int grid_for(long long n, int per_block, int max_blocks = AMG_MAX_BLOCKS) {
  long long g = (n + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > max_blocks) g = max_blocks;
  return (int)g;
}

// ---------------------------------------------------------------------------
// Shared device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of NV per-thread values over the block, fixed tree order; result valid in
// thread 0.  sh must hold NV * 32 doubles.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double *sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k * 32 + wid] = v[k];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = lane < nw ? sh[k * 32 + lane] : 0.0;
      v[k] = warp_sum(s);
    }
  }
  __syncthreads();
}

// Deterministic grid reduction: every block stores its NV partial sums in
// part[k * gridDim.x + blockIdx.x]; the last block to arrive (by an atomic
// counter) sums the partials in index order and returns true with the totals
// in `tot` (valid in thread 0 of that block).  The counter is reset for reuse.
template <int NV>
__device__ __forceinline__ bool grid_sum_last(double (&v)[NV], double *part, unsigned *counter,
                                              double (&tot)[NV]) {
  __shared__ double sh[NV * 32];
  __shared__ bool last;
  block_sum<NV>(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) part[k * gridDim.x + blockIdx.x] = v[k];
    __threadfence();
    unsigned prev = atomicAdd(counter, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double s[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    s[k] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
      s[k] += __ldcg(&part[k * gridDim.x + b]);
  }
  block_sum<NV>(s, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) tot[k] = s[k];
    *counter = 0u;
  }
  return true;
}

#define BARRIER_SPIN_LIMIT (1ll << 31)  // clock cycles (about one second)

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Monotonic-counter grid barrier: the k-th barrier completes when the counter
// reaches k * G.  Waits are bounded; a block that gives up sets the timeout
// flag and the caller leaves its loop.  arrive() and wait() may be split so
// that a block does independent work while the others arrive.
struct GridBarrier {
  unsigned *count;
  unsigned target;
  long long limit = BARRIER_SPIN_LIMIT;
  unsigned sleep_ns = 0;  // pause between polls (0: poll continuously)
  __device__ __forceinline__ void arrive(unsigned G) {
    __syncthreads();
    target += G;
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(count, 1u);
    }
  }
  __device__ __forceinline__ bool wait(unsigned *eflags, int *fail_sh) {
    if (threadIdx.x == 0) {
      long long t0 = clock64();
      while (ld_acquire_u32(count) < target) {
        if (sleep_ns) __nanosleep(sleep_ns);
        if (clock64() - t0 > limit) {
          atomicOr(eflags, AMG_EFLAG_TIMEOUT);
          *fail_sh = 1;
          break;
        }
      }
    }
    __syncthreads();
    return *fail_sh == 0;
  }
  __device__ __forceinline__ bool sync(unsigned G, unsigned *eflags, int *fail_sh) {
    arrive(G);
    return wait(eflags, fail_sh);
  }
};

__device__ __forceinline__ bool is_done(const KState *st) {
  return st != nullptr && *((volatile const int *)&st->done) != 0;
}

// ---------------------------------------------------------------------------
// Cross-TU host entry points
// ---------------------------------------------------------------------------
// V-cycle of level `k` with right-hand side f and output x (FP64 or FP32 per
// the hierarchy's precision); `st` may be a Krylov state whose done flag
// turns every kernel into a no-op.
amg_status vcycle_run(amg_hierarchy *h, const double *r, double *z, cudaStream_t s, const KState *st);
amg_status coarse_setup(amg_hierarchy *h, cudaStream_t s);
amg_status dense_inverse(amg_hierarchy *h, cudaStream_t s);
template <typename T>
amg_status dense_refined_solve(amg_hierarchy *h, const T *f, T *x, int steps, cudaStream_t s, const KState *st);
amg_status precision_setup(amg_hierarchy *h, cudaStream_t s);
amg_status operator_form_setup(amg_hierarchy *h, cudaStream_t s);
void reset_graphs(amg_hierarchy *h);
amg_status cluster_cg_config(int n, ClusterCG *cc);
template <typename T>
amg_status cluster_cg_launch(const ClusterCG &cc, int n, const int32_t *rp, const int32_t *ci, const double *val,
                             const double *dinv, const T *f, T *x, int *iters, unsigned long long *iters_total,
                             const KState *st, cudaStream_t s);
amg_status read_eflags(amg_hierarchy *h, cudaStream_t s, unsigned *flags);
#ifndef CG_THREADS
#define CG_THREADS 512
#endif
#define CG_PART_DOUBLES (6 * AMG_MAX_BLOCKS + 32)
#define CG_SMEM_CAP (200 * 1024)
// Grid, block and shared-memory configuration of the coarse CG for n rows on
// the current device (also sets the kernel's shared-memory limit).
amg_status coarse_cg_config(int n, CoarseCG *cg);
amg_status coarse_cg_prepare(int n, const int32_t *rp, const CoarseCG &cg, cudaStream_t s);
amg_status coarse_cg_launch(int n, const int32_t *rp, const int32_t *ci, const double *val, const double *dinv,
                            const double *f, double *x, const CoarseCG &cg, unsigned *eflags, cudaStream_t s);
