// noalloc.cu -- a coarse-solver entry point that performs no device allocation.
//
// Some callers cannot call cudaMalloc: plugins hosted by a framework that owns
// all device memory and forbids allocations outside its own pool, and
// latency-critical host loops that must not take cudaMalloc's implicit device
// synchronisation.  For them, amg_coarse_cg_noalloc runs the library's
// Jacobi-PCG solver with every work vector in one fixed array compiled into
// the library (below), so a call allocates nothing.  The price: every GPU
// that loads the library holds this array until the process exits, sizes are
// capped, and all calls share it.
#include <cmath>
#include <mutex>

#include "common.cuh"

// Largest system accepted: 262,144 rows and 2^31 - 1 stored entries.
#define NOALLOC_MAX_N 262144
#define NOALLOC_CG_MAXIT 1000    // the solver's iteration limit
#define NOALLOC_CONVERGED 1e-10  // recomputed relative residual accepted as converged
#define NOALLOC_ALIGN 256
#define NOALLOC_VECS 14  // dinv, the solver's twelve work vectors and the row order
#define NOALLOC_BYTES                                                                            \
  ((size_t)NOALLOC_VECS * 8 * (NOALLOC_MAX_N + AMG_PAD) + (size_t)CG_PART_DOUBLES * 8 + \
   (size_t)5 * AMG_MAX_BLOCKS * 4 + 16 * NOALLOC_ALIGN)

// The scratch array: about 29 MB on every device that loads the library.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

namespace {

std::mutex g_noalloc_mu;
void *g_noalloc_base[256] = {nullptr};  // device address of the array, per device ordinal

size_t up(size_t v) { return (v + NOALLOC_ALIGN - 1) / NOALLOC_ALIGN * NOALLOC_ALIGN; }

// Device address of the scratch array on the current device (looked up once per
// device; the array's host-side name is not a device address).
amg_status scratch_base(unsigned char **out) {
  int dev = 0;
  AMG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return AMG_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_base[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return amg_cuda_status(e != cudaSuccess ? e : cudaErrorInvalidSymbol);
    }
    g_noalloc_base[dev] = p;
  }
  *out = (unsigned char *)g_noalloc_base[dev];
  return AMG_OK;
}

// CSR checks and 1/a_ii into the scratch; flags[0] collects error bits.
__global__ void k_noalloc_prepare(int n, long long nnz, const int32_t *__restrict__ rp,
                                  const int32_t *__restrict__ ci, const double *__restrict__ val,
                                  double *__restrict__ dinv, unsigned *flags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && (rp[0] != 0 || (long long)rp[n] != nnz)) atomicOr(flags, AMG_EFLAG_BAD_CSR);
  if (i >= n) return;
  int b = rp[i], e = rp[i + 1];
  if (b < 0 || e < b || (long long)e > nnz) { atomicOr(flags, AMG_EFLAG_BAD_CSR); dinv[i] = 0.0; return; }
  double d = 0.0;
  int prev = -1;
  for (int k = b; k < e; ++k) {
    int c = ci[k];
    if (c < 0 || c >= n || c <= prev) { atomicOr(flags, AMG_EFLAG_BAD_CSR); dinv[i] = 0.0; return; }
    prev = c;
    if (c == i) d = val[k];
  }
  if (d == 0.0 || !isfinite(d)) { atomicOr(flags, AMG_EFLAG_ZERO_DIAG); dinv[i] = 0.0; return; }
  dinv[i] = 1.0 / d;
}

// Partial sums of ||f - A x||^2 and ||f||^2 per block (fixed order), for the
// status of the solve.
__global__ void k_noalloc_resid(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                const double *__restrict__ val, const double *__restrict__ f,
                                const double *__restrict__ x, double *__restrict__ part) {
  __shared__ double sh[2 * 32];
  double v[2] = {0.0, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double ax = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) ax += val[k] * x[ci[k]];
    const double r = f[i] - ax;
    v[0] += r * r;
    v[1] += f[i] * f[i];
  }
  block_sum<2>(v, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = v[0];
    part[gridDim.x + blockIdx.x] = v[1];
  }
}

// out[0..1] = the sums of the block partials, in block order (one thread).
__global__ void k_noalloc_total(int blocks, const double *__restrict__ part, double *__restrict__ out) {
  double a = 0.0, b = 0.0;
  for (int k = 0; k < blocks; ++k) {
    a += part[k];
    b += part[blocks + k];
  }
  out[0] = a;
  out[1] = b;
}

}  // namespace

extern "C" amg_status amg_coarse_cg_noalloc(int n, int64_t nnz, const int32_t *d_row_ptr, const int32_t *d_col,
                                            const double *d_val, const double *d_f, double *d_x,
                                            amg_stream_t stream, int *iterations) {
  clear_stale_cuda_error();
  if (iterations) *iterations = 0;
  if (n <= 0 || n > NOALLOC_MAX_N || nnz < 0 || nnz >= (1ll << 31) || !d_row_ptr || !d_f || !d_x ||
      (const void *)d_f == (const void *)d_x || (nnz > 0 && (!d_col || !d_val)))
    return AMG_ERR_INVALID_ARG;
  unsigned char *base = nullptr;
  AMG_TRY(scratch_base(&base));
  cudaStream_t s = (cudaStream_t)stream;
  // carve the array: vectors, reduction partials, barrier words, counters
  const size_t vb = up(sizeof(double) * ((size_t)n + AMG_PAD));
  size_t off = 0;
  auto take = [&](size_t bytes) { unsigned char *p = base + off; off += up(bytes); return p; };
  double *dinv = (double *)take(vb);
  CoarseCG cg;
  cg.n = n;
  cg.halo[0] = (double *)take(vb);
  cg.halo[1] = (double *)take(vb);
  cg.state = (double *)take(vb * CG_STATE);
  cg.part = (double *)take(sizeof(double) * CG_PART_DOUBLES);
  cg.ord = (int *)take(sizeof(int) * ((size_t)n + AMG_PAD));
  cg.meta = (int *)take(sizeof(int) * 5 * AMG_MAX_BLOCKS);
  cg.bar = (unsigned *)take(sizeof(unsigned) * 4);
  cg.iters = (int *)take(sizeof(int) * 4);
  cg.iters_total = (unsigned long long *)take(sizeof(unsigned long long));
  unsigned *flags = (unsigned *)take(sizeof(unsigned) * 4);
  double *norms = (double *)take(sizeof(double) * 2);
  if (off > NOALLOC_BYTES) return AMG_ERR_UNSUPPORTED;
  AMG_TRY(coarse_cg_config(n, &cg));
  // the array keeps the previous call's contents: clear what must start at zero
  AMG_CUDA(cudaMemsetAsync(flags, 0, sizeof(unsigned) * 4, s));
  AMG_CUDA(cudaMemsetAsync(cg.iters_total, 0, sizeof(unsigned long long), s));
  k_noalloc_prepare<<<cdiv(n, AMG_THREADS), AMG_THREADS, 0, s>>>(n, nnz, d_row_ptr, d_col, d_val, dinv, flags);
  count_launch();
  AMG_CUDA(cudaGetLastError());
  unsigned hflags[2] = {0, 0};
  AMG_CUDA(cudaMemcpyAsync(hflags, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  AMG_CUDA(cudaStreamSynchronize(s));
  if (hflags[0] & AMG_EFLAG_BAD_CSR) return AMG_ERR_INVALID_CSR;
  if (hflags[0] & AMG_EFLAG_ZERO_DIAG) return AMG_ERR_ZERO_DIAG;
  AMG_TRY(coarse_cg_prepare(n, d_row_ptr, cg, s));
  AMG_TRY(coarse_cg_launch(n, d_row_ptr, d_col, d_val, dinv, d_f, d_x, cg, flags, s));
  // residual recomputed from x (the reduction partials reuse the solver's)
  const int rblocks = std::min(cdiv(n, AMG_THREADS), 2 * AMG_MAX_BLOCKS);
  k_noalloc_resid<<<rblocks, AMG_THREADS, 0, s>>>(n, d_row_ptr, d_col, d_val, d_f, d_x, cg.part);
  k_noalloc_total<<<1, 1, 0, s>>>(rblocks, cg.part, norms);
  count_launch(2);
  AMG_CUDA(cudaGetLastError());
  int it = 0;
  double hn[2] = {0.0, 0.0};
  AMG_CUDA(cudaMemcpyAsync(hflags, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  AMG_CUDA(cudaMemcpyAsync(&it, cg.iters, sizeof(int), cudaMemcpyDeviceToHost, s));
  AMG_CUDA(cudaMemcpyAsync(hn, norms, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
  AMG_CUDA(cudaStreamSynchronize(s));
  if (iterations) *iterations = it;
  if (hflags[0] & AMG_EFLAG_TIMEOUT) return AMG_ERR_TIMEOUT;
  if (!std::isfinite(hn[0]) || !std::isfinite(hn[1])) return AMG_ERR_BREAKDOWN;
  // the solver stops at a recurrence residual of 1e-12 ||f||; the recomputed
  // one may sit a little above that, so convergence is judged at 1e-10
  if (it >= NOALLOC_CG_MAXIT || std::sqrt(hn[0]) > NOALLOC_CONVERGED * std::sqrt(hn[1]))
    return AMG_ERR_NOT_CONVERGED;
  return AMG_OK;
}
