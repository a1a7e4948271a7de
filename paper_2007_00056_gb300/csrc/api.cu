// api.cu -- small C-ABI entry points and host helpers shared by the library.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "common.cuh"

unsigned long long g_amg_launches = 0;

void prof_begin(amg_hierarchy *h, cudaStream_t s, int id, double bytes) {
  Profiler &p = h->prof;
  if (p.pool.size() < 2) {
    for (int k = 0; k < 64; ++k) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return; }
      p.pool.push_back(e);
    }
  }
  Profiler::Rec r;
  r.id = id;
  r.bytes = bytes;
  r.a = p.pool.back(); p.pool.pop_back();
  r.b = p.pool.back(); p.pool.pop_back();
  cudaEventRecord(r.a, s);
  p.pending.push_back(r);
}

void prof_end(amg_hierarchy *h, cudaStream_t s) {
  Profiler &p = h->prof;
  if (!p.pending.empty()) cudaEventRecord(p.pending.back().b, s);
}

// Accumulates the timings of every recorded launch (waits for them).
amg_status prof_flush(amg_hierarchy *h) {
  Profiler &p = h->prof;
  for (auto &r : p.pending) {
    cudaEventSynchronize(r.b);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess && r.id >= 0 && r.id < AMG_PROF_IDS) {
      p.ms[r.id] += ms;
      p.bytes[r.id] += r.bytes;
      p.launches[r.id] += 1;
    }
    cudaGetLastError();
    p.pool.push_back(r.a);
    p.pool.push_back(r.b);
  }
  p.pending.clear();
  return AMG_OK;
}

static thread_local cudaError_t g_last_cuda_error = cudaSuccess;

static thread_local const char *g_last_cuda_file = nullptr;
static thread_local int g_last_cuda_line = 0;

amg_status amg_cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return AMG_OK;
  g_last_cuda_error = e;
  g_last_cuda_file = nullptr;
  if (e == cudaErrorMemoryAllocation) return AMG_ERR_OOM;
  return AMG_ERR_CUDA;
}

amg_status amg_cuda_status_at(cudaError_t e, const char *file, int line) {
  const amg_status s = amg_cuda_status(e);
  if (s != AMG_OK) {
    const char *base = strrchr(file, '/');
    g_last_cuda_file = base ? base + 1 : file;
    g_last_cuda_line = line;
  }
  return s;
}

namespace {
std::mutex g_pool_mu;
cudaMemPool_t g_pool[256] = {nullptr};

// The library's memory pool on the current device, created on first use with
// a release threshold that keeps freed blocks for reuse by later setups.
cudaMemPool_t lib_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) { cudaGetLastError(); return nullptr; }
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    // a block freed on one stream is not handed to another stream by making
    // that stream wait for the first: setups on different streams stay
    // independent (the pool takes fresh memory instead)
    int no = 0;
    cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
    g_pool[dev] = pool;
  }
  return g_pool[dev];
}
}  // namespace

amg_status pool_alloc(void **p, size_t bytes, cudaStream_t s) {
  cudaMemPool_t pool = lib_pool();
  cudaError_t e = pool ? cudaMallocFromPoolAsync(p, bytes ? bytes : 16, pool, s) : cudaMalloc(p, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return AMG_ERR_OOM;
  }
  return AMG_OK;
}

void pool_free(void *p, cudaStream_t s) {
  if (p && cudaFreeAsync(p, s) != cudaSuccess) cudaGetLastError();
}

void pool_trim() {
  cudaMemPool_t pool = lib_pool();
  if (pool && cudaMemPoolTrimTo(pool, 0) != cudaSuccess) cudaGetLastError();
}

// Small pinned host buffers (<= 256 bytes) for device-to-host status reads,
// carved from 64 KB pinned chunks and recycled, so a setup pays no
// cudaMallocHost.
namespace {
std::mutex g_pin_mu;
std::vector<void *> g_pin_free;
}  // namespace

void *pinned_small_alloc() {
  std::lock_guard<std::mutex> lock(g_pin_mu);
  if (g_pin_free.empty()) {
    void *chunk = nullptr;
    if (cudaMallocHost(&chunk, 65536) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    for (int k = 0; k < 256; ++k) g_pin_free.push_back((char *)chunk + 256 * k);
  }
  void *p = g_pin_free.back();
  g_pin_free.pop_back();
  memset(p, 0, 256);
  return p;
}

void pinned_small_free(void *p) {
  if (!p) return;
  std::lock_guard<std::mutex> lock(g_pin_mu);
  g_pin_free.push_back(p);
}

amg_status hier_alloc(amg_hierarchy *h, void **p, size_t bytes) {
  AMG_TRY(pool_alloc(p, bytes, h->stream));
  h->allocs.push_back({*p, bytes});
  return AMG_OK;
}

// Reads and clears the device error bits (synchronises the stream).
amg_status read_eflags(amg_hierarchy *h, cudaStream_t s, unsigned *flags) {
  AMG_CUDA(cudaMemcpyAsync(h->eflags_host, h->eflags, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  AMG_CUDA(cudaStreamSynchronize(s));
  *flags = h->eflags_host[0];
  if (*flags) AMG_CUDA(cudaMemsetAsync(h->eflags, 0, sizeof(unsigned), s));
  return AMG_OK;
}

extern "C" amg_status amg_default_params(amg_params *p) {
  if (!p) return AMG_ERR_INVALID_ARG;
  p->passes = 2;
  p->max_levels = 10;
  p->coarse_max = 4096;
  p->stall_ratio = 0.85;
  p->omega = 2.0 / 3.0;
  p->nu_pre = 1;
  p->nu_post = 1;
  p->coarse_solver = AMG_COARSE_AUTO;
  p->precision = AMG_FP64;
  p->cycle = AMG_CYCLE_V;
  p->tie_break = AMG_TIE_SMALLER;
  p->edge_weight = AMG_WEIGHT_ABS;
  p->operator_form = 1;
  p->dense_max = 0;
  p->graphs = 0;
  return AMG_OK;
}

extern "C" const char *amg_last_cuda_error(void) {
  static thread_local char text[256];
  if (g_last_cuda_error == cudaSuccess) return "no CUDA error";
  if (!g_last_cuda_file) return cudaGetErrorString(g_last_cuda_error);
  snprintf(text, sizeof(text), "%s (at %s:%d)", cudaGetErrorString(g_last_cuda_error), g_last_cuda_file,
           g_last_cuda_line);
  return text;
}

extern "C" const char *amg_status_string(amg_status s) {
  switch (s) {
    case AMG_OK: return "ok";
    case AMG_ERR_INVALID_ARG: return "invalid argument";
    case AMG_ERR_INVALID_CSR: return "invalid CSR structure";
    case AMG_ERR_ZERO_DIAG: return "zero or missing diagonal entry";
    case AMG_ERR_OOM: return "device out of memory";
    case AMG_ERR_BREAKDOWN: return "Krylov breakdown";
    case AMG_ERR_NOT_CONVERGED: return "not converged within max_iter";
    case AMG_ERR_TIMEOUT: return "bounded device wait timed out";
    case AMG_ERR_CUDA: return "CUDA runtime error";
    case AMG_ERR_UNSUPPORTED: return "unsupported input or option";
  }
  return "unknown status";
}

extern "C" int amg_num_levels(const amg_hierarchy *h) { return h ? h->L + 1 : -1; }

extern "C" amg_status amg_level_info(const amg_hierarchy *h, int level, int *n, int64_t *nnz, int32_t *d_agg_out,
                                     amg_stream_t stream) {
  clear_stale_cuda_error();
  if (!h || level < 0 || level > h->L) return AMG_ERR_INVALID_ARG;
  if (d_agg_out && level == h->L) return AMG_ERR_INVALID_ARG;
  const Level &l = h->lev[level];
  if (n) *n = l.n;
  if (nnz) *nnz = l.nnz;
  cudaStream_t s = (cudaStream_t)stream;
  if (d_agg_out) {
    AMG_CUDA(cudaMemcpyAsync(d_agg_out, l.agg, sizeof(int32_t) * l.n, cudaMemcpyDeviceToDevice, s));
    AMG_CUDA(cudaStreamSynchronize(s));
  }
  return AMG_OK;
}

extern "C" amg_status amg_export_level(const amg_hierarchy *h, int level, int32_t *d_row_ptr, int32_t *d_col,
                                       double *d_val, amg_stream_t stream) {
  clear_stale_cuda_error();
  if (!h || level < 0 || level > h->L || !d_row_ptr) return AMG_ERR_INVALID_ARG;
  const Level &l = h->lev[level];
  if (l.nnz > 0 && (!d_col || !d_val)) return AMG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  AMG_CUDA(cudaMemcpyAsync(d_row_ptr, l.rp, sizeof(int32_t) * (l.n + 1), cudaMemcpyDeviceToDevice, s));
  if (l.nnz > 0) {
    AMG_CUDA(cudaMemcpyAsync(d_col, l.ci, sizeof(int32_t) * l.nnz, cudaMemcpyDefault, s));
    AMG_CUDA(cudaMemcpyAsync(d_val, l.val, sizeof(double) * l.nnz, cudaMemcpyDefault, s));
  }
  AMG_CUDA(cudaStreamSynchronize(s));
  return AMG_OK;
}

extern "C" void amg_destroy(amg_hierarchy *h) {
  if (!h) return;
  // wait for the latest work that used the hierarchy (its calls are otherwise
  // synchronous), not for the whole device: other streams keep running
  cudaStreamSynchronize(h->last_stream ? h->last_stream : h->stream);
  cudaGetLastError();
  if (h->g_vcycle) cudaGraphExecDestroy(h->g_vcycle);
  if (h->g_pcg) cudaGraphExecDestroy(h->g_pcg);
  if (h->g_bicg) cudaGraphExecDestroy(h->g_bicg);
  if (h->g_amg) cudaGraphExecDestroy(h->g_amg);
  prof_flush(h);
  for (cudaEvent_t e : h->prof.pool) cudaEventDestroy(e);
  // stream-ordered frees back into the library pool, on the hierarchy's own stream
  residency_release(h);
  for (auto &a : h->allocs) pool_free(a.first, h->cap_stream);
  pinned_small_free(h->st_host);
  pinned_small_free(h->eflags_host);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  cudaGetLastError();
  delete h;
}

extern "C" int amg_coarse_cg_cluster_size(const amg_hierarchy *h) {
  if (!h || h->dense) return -1;
  return h->cg.cl.size;
}

extern "C" unsigned long long amg_kernel_launches(void) { return __atomic_load_n(&g_amg_launches, __ATOMIC_RELAXED); }

extern "C" amg_status amg_profile_enable(amg_hierarchy *h, int on) {
  if (!h) return AMG_ERR_INVALID_ARG;
  prof_flush(h);
  h->prof.on = on != 0;
  return AMG_OK;
}

extern "C" amg_status amg_profile_reset(amg_hierarchy *h) {
  if (!h) return AMG_ERR_INVALID_ARG;
  prof_flush(h);
  for (int i = 0; i < AMG_PROF_IDS; ++i) { h->prof.ms[i] = 0; h->prof.bytes[i] = 0; h->prof.launches[i] = 0; }
  if (h->cg.iters_total) cudaMemset(h->cg.iters_total, 0, sizeof(unsigned long long));
  return AMG_OK;
}

extern "C" amg_status amg_profile_read(amg_hierarchy *h, int kind, int level, double *ms, double *bytes,
                                       long long *launches) {
  if (!h || kind < 0 || kind >= PK_COUNT || level < 0 || level >= AMG_MAX_LEVELS) return AMG_ERR_INVALID_ARG;
  prof_flush(h);
  int id = kind * AMG_MAX_LEVELS + level;
  double b = h->prof.bytes[id];
  if (kind == PK_COARSE_CG && h->cg.iters_total) {
    // bytes of the coarse CG depend on its iteration count, summed on the device
    unsigned long long it = 0;
    cudaMemcpy(&it, h->cg.iters_total, sizeof(it), cudaMemcpyDeviceToHost);
    b = h->prof.launches[id] > 0 ? (double)it * (h->prof.bytes[id] / (double)h->prof.launches[id]) : 0.0;
  }
  if (ms) *ms = h->prof.ms[id];
  if (bytes) *bytes = b;
  if (launches) *launches = h->prof.launches[id];
  return AMG_OK;
}
