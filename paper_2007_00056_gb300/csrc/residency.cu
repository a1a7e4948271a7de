// residency.cu -- level matrices kept in host memory during the solve phase.
//
// The hybrid CPU/GPU-CI algorithm (Sec. 3.1.1) rests on one observation: a
// multigrid cycle works on one level at a time, so only that level's
// matrices need to be in device memory; the others can wait in host memory
// and be copied in when the cycle reaches them, the copy of the next level
// overlapping the kernels of the current one on a second stream.
//
// On GB300 the host memory sits behind the coherent NVLink-C2C link, so two
// forms are offered:
//   AMG_HOST_MAPPED  the arrays live in pinned host memory and the kernels
//                    read them there: every matrix pass of such a level
//                    streams its bytes over the link (no device copy at all);
//   AMG_HOST_STAGED  the paper's scheme: each cycle visit of such a level
//                    reads its matrix from one of two device buffers, filled
//                    by cudaMemcpyAsync on a copy stream; while a visit runs,
//                    the copy for the visit predicted next fills the other
//                    buffer.  The prediction follows the V-cycle order
//   (descending visits k = first..L-1, then ascending L-1..first, then the
// next cycle's first descending visit); a visit it did not predict (W- and
// F-cycles) is copied on demand, so every cycle kind stays correct.
//
// What moves: for each level k >= first (below the coarsest), the arrays
// whose length is the number of nonzeros: column indices and values of A, of
// its FP32 / FP16 copies, of C = I - omega A D^-1 and of Q = P - omega D^-1 A P
// (pattern and values).  Everything of length n (row pointers, diagonals,
// aggregate maps, vectors) stays in device memory.  With AMG_HOST_STAGED the
// level-0 matrix A itself stays in device memory: the outer Krylov method
// multiplies by it every iteration.
#include "common.cuh"

#include <cstddef>
#include <cstring>

namespace {

// A matrix array of a level, by its field in Level.
struct Field {
  size_t off;       // offsetof(Level, field)
  size_t elem;      // element size
  int len;          // 0: nnz + AMG_PAD elements, 1: qnnz + AMG_PAD elements
};

#define FIELD(name, type, len) Field{offsetof(Level, name), sizeof(type), len}
const Field kFields[] = {
    FIELD(ci, int32_t, 0),   FIELD(val, double, 0),  FIELD(val32, float, 0),   FIELD(val16, __half, 0),
    FIELD(cval, double, 0),  FIELD(cval32, float, 0), FIELD(qci, int32_t, 1),  FIELD(qval, double, 1),
    FIELD(qval32, float, 1),
};
#undef FIELD
constexpr int kNumFields = (int)(sizeof(kFields) / sizeof(kFields[0]));

void *&field_ref(Level &l, const Field &f) { return *reinterpret_cast<void **>(reinterpret_cast<char *>(&l) + f.off); }
size_t field_bytes(const Level &l, const Field &f) {
  return f.elem * (size_t)((f.len == 0 ? l.nnz : l.qnnz) + AMG_PAD);
}

// The arrays one visit reads, for the hierarchy's precision (fields by index
// into kFields; -1 ends the list).
void set_fields(const amg_hierarchy *h, int set, int out[2]) {
  const int p = h->prm.precision;
  out[0] = out[1] = -1;
  switch (set) {
    case SET_A: out[0] = 0; out[1] = p == AMG_FP64 ? 1 : p == AMG_FP32 ? 2 : 3; break;
    case SET_C: out[0] = 0; out[1] = p == AMG_FP64 ? 4 : 5; break;
    case SET_Q: out[0] = 6; out[1] = p == AMG_FP64 ? 7 : 8; break;
    default: break;
  }
}

}  // namespace

// Two device buffers, their fill and release events, and what each holds.
struct Stager {
  cudaStream_t copy = nullptr;
  char *slot[2] = {nullptr, nullptr};
  size_t slot_bytes = 0;
  cudaEvent_t ready[2] = {nullptr, nullptr};  // recorded on `copy` after a fill
  cudaEvent_t freed[2] = {nullptr, nullptr};  // recorded on the compute stream after a visit's kernels
  int key[2] = {-1, -1};                      // 3 k + set held (or being filled) by each slot
  int cur = -1;                               // slot of the visit between acquire and release
  int last = 1;                               // slot of the latest released visit
  // per level and set: the host arrays and their offsets within a slot
  int nf[AMG_MAX_LEVELS][3] = {};
  int fid[AMG_MAX_LEVELS][3][2] = {};
  size_t soff[AMG_MAX_LEVELS][3][2] = {};
  unsigned long long copied = 0, fills = 0, visits = 0;
};

namespace {

bool is_host(const amg_hierarchy *h, const void *p) {
  for (const auto &a : h->host_allocs)
    if (a.first == p) return true;
  return false;
}

// The zero-guess visit of level k uses the residual-operator form.
bool op_visit(const amg_hierarchy *h, int k) {
  const Level &l = h->lev[k];
  if (!l.op_on || h->prm.nu_pre != 1 || h->prm.nu_post != 1) return false;
  if (h->prm.precision == AMG_FP64) return l.cval != nullptr;
  if (h->prm.precision == AMG_FP32) return l.cval32 != nullptr;
  return false;
}
int down_set(const amg_hierarchy *h, int k) { return op_visit(h, k) ? SET_C : SET_A; }
int up_set(const amg_hierarchy *h, int k) {
  if (op_visit(h, k)) return SET_Q;
  return h->prm.nu_post > 0 ? SET_A : SET_NONE;
}

// The visit after (k, descending?) in V-cycle order, over host-resident
// levels; false if there is none with arrays to copy.
bool predict_next(const amg_hierarchy *h, int k, bool descending, int *nk, int *nset) {
  const int first = h->res_first, L = h->L;
  if (descending) {
    if (k + 1 < L) { *nk = k + 1; *nset = down_set(h, k + 1); return true; }
    // the coarsest level is solved in device memory; then level k ascends
    for (int j = k; j >= first; --j) {
      const int s = up_set(h, j);
      if (s != SET_NONE) { *nk = j; *nset = s; return true; }
    }
  } else {
    for (int j = k - 1; j >= first; --j) {
      const int s = up_set(h, j);
      if (s != SET_NONE) { *nk = j; *nset = s; return true; }
    }
  }
  if (first >= L) return false;
  *nk = first;  // the next cycle starts by descending into `first`
  *nset = down_set(h, first);
  return true;
}

void fill_slot(amg_hierarchy *h, int x, int k, int set) {
  Stager &g = *h->stg;
  const Level &l = h->lev[k];
  cudaStreamWaitEvent(g.copy, g.freed[x], 0);
  for (int i = 0; i < g.nf[k][set]; ++i) {
    const Field &f = kFields[g.fid[k][set][i]];
    const void *src = field_ref(const_cast<Level &>(l), f);
    const size_t bytes = field_bytes(l, f);
    cudaMemcpyAsync(g.slot[x] + g.soff[k][set][i], src, bytes, cudaMemcpyHostToDevice, g.copy);
    g.copied += bytes;
  }
  cudaEventRecord(g.ready[x], g.copy);
  g.key[x] = 3 * k + set;
  g.fills += 1;
}

// Moves one array between device and pinned host memory (the hierarchy's
// bookkeeping follows it).  The stream is synchronised before the old copy is
// freed.
amg_status move_array(amg_hierarchy *h, void *&ptr, size_t bytes, bool to_host, cudaStream_t s) {
  if (!ptr) return AMG_OK;
  void *old = ptr;
  void *fresh = nullptr;
  if (to_host) {
    if (cudaHostAlloc(&fresh, bytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
      cudaGetLastError();
      return AMG_ERR_OOM;
    }
  } else {
    AMG_TRY(pool_alloc(&fresh, bytes, s));
  }
  cudaError_t e = cudaMemcpyAsync(fresh, old, bytes, cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    if (to_host) cudaFreeHost(fresh); else pool_free(fresh, s);
    return amg_cuda_status(e);
  }
  if (to_host) {
    void *dptr = nullptr;
    if (cudaHostGetDevicePointer(&dptr, fresh, 0) != cudaSuccess || dptr != fresh) {
      // the library relies on unified addressing: the host pointer is the device pointer
      cudaGetLastError();
      cudaFreeHost(fresh);
      return AMG_ERR_UNSUPPORTED;
    }
    for (size_t i = 0; i < h->allocs.size(); ++i)
      if (h->allocs[i].first == old) { h->allocs.erase(h->allocs.begin() + (long)i); break; }
    pool_free(old, s);
    h->host_allocs.push_back({fresh, bytes});
  } else {
    for (size_t i = 0; i < h->host_allocs.size(); ++i)
      if (h->host_allocs[i].first == old) { h->host_allocs.erase(h->host_allocs.begin() + (long)i); break; }
    cudaFreeHost(old);
    h->allocs.push_back({fresh, bytes});
  }
  ptr = fresh;
  return AMG_OK;
}

void stager_free(amg_hierarchy *h) {
  Stager *g = h->stg;
  if (!g) return;
  if (g->copy) cudaStreamSynchronize(g->copy);
  for (int x = 0; x < 2; ++x) {
    if (g->slot[x]) cudaFree(g->slot[x]);
    if (g->ready[x]) cudaEventDestroy(g->ready[x]);
    if (g->freed[x]) cudaEventDestroy(g->freed[x]);
  }
  if (g->copy) cudaStreamDestroy(g->copy);
  cudaGetLastError();
  delete g;
  h->stg = nullptr;
}

amg_status stager_create(amg_hierarchy *h) {
  Stager *g = new Stager();
  h->stg = g;
  size_t need = 0;
  for (int k = 0; k < h->L; ++k) {
    const Level &l = h->lev[k];
    if (!l.host) continue;
    for (int set = 0; set < 3; ++set) {
      int ids[2];
      set_fields(h, set, ids);
      size_t off = 0;
      int n = 0;
      for (int i = 0; i < 2; ++i) {
        if (ids[i] < 0) continue;
        const Field &f = kFields[ids[i]];
        const void *p = field_ref(const_cast<Level &>(l), f);
        if (!p || !is_host(h, p)) continue;  // absent, or kept in device memory
        g->fid[k][set][n] = ids[i];
        g->soff[k][set][n] = off;
        off += (field_bytes(l, f) + 255) / 256 * 256;
        ++n;
      }
      g->nf[k][set] = n;
      need = std::max(need, off);
    }
  }
  g->slot_bytes = need;
  if (cudaStreamCreateWithFlags(&g->copy, cudaStreamNonBlocking) != cudaSuccess) goto cuda_fail;
  for (int x = 0; x < 2; ++x) {
    if (need && cudaMalloc(&g->slot[x], need) != cudaSuccess) { cudaGetLastError(); stager_free(h); return AMG_ERR_OOM; }
    if (cudaEventCreateWithFlags(&g->ready[x], cudaEventDisableTiming) != cudaSuccess) goto cuda_fail;
    if (cudaEventCreateWithFlags(&g->freed[x], cudaEventDisableTiming) != cudaSuccess) goto cuda_fail;
    if (cudaEventRecord(g->ready[x], g->copy) != cudaSuccess) goto cuda_fail;
    if (cudaEventRecord(g->freed[x], g->copy) != cudaSuccess) goto cuda_fail;
  }
  return AMG_OK;
cuda_fail:
  {
    const cudaError_t e = cudaGetLastError();
    stager_free(h);
    return amg_cuda_status(e);
  }
}

// Moves the matrix arrays of levels [first, L) to host memory (or all back).
amg_status move_levels(amg_hierarchy *h, int first, bool to_host, bool keep_a0, cudaStream_t s) {
  for (int k = first; k < h->L; ++k) {
    Level &l = h->lev[k];
    for (int i = 0; i < kNumFields; ++i) {
      const Field &f = kFields[i];
      if (to_host && keep_a0 && k == 0 && (i == 0 || i == 1)) continue;  // the Krylov method's A
      void *&p = field_ref(l, f);
      if (!p || is_host(h, p) == to_host) continue;
      AMG_TRY(move_array(h, p, field_bytes(l, f), to_host, s));
    }
    if (to_host && !l.host) {
      l.st_cap_dev = l.st_cap;
      l.st_cap = 0;  // the TMA-staged row kernels read device memory only
      l.host = 1;
    } else if (!to_host && l.host) {
      l.st_cap = l.st_cap_dev;
      l.host = 0;
    }
  }
  return AMG_OK;
}

}  // namespace

void reset_graphs(amg_hierarchy *h);

Level stage_acquire(amg_hierarchy *h, int k, int set, cudaStream_t s) {
  Stager &g = *h->stg;
  Level lv = h->lev[k];
  g.cur = -1;
  if (set < 0 || set > 2 || g.nf[k][set] == 0) return lv;
  const int key = 3 * k + set;
  int x = g.key[0] == key ? 0 : g.key[1] == key ? 1 : -1;
  if (x < 0) {
    x = 1 - g.last;  // keep the latest visit's buffer: it may be read again next
    fill_slot(h, x, k, set);
  }
  cudaStreamWaitEvent(s, g.ready[x], 0);
  for (int i = 0; i < g.nf[k][set]; ++i) field_ref(lv, kFields[g.fid[k][set][i]]) = g.slot[x] + g.soff[k][set][i];
  g.cur = x;
  g.visits += 1;
  return lv;
}

void stage_release(amg_hierarchy *h, int k, bool descending, cudaStream_t s) {
  Stager &g = *h->stg;
  if (g.cur >= 0) {
    cudaEventRecord(g.freed[g.cur], s);
    g.last = g.cur;
    g.cur = -1;
  }
  int nk = 0, nset = SET_NONE;
  if (!predict_next(h, k, descending, &nk, &nset) || nset == SET_NONE || g.nf[nk][nset] == 0) return;
  const int key = 3 * nk + nset;
  if (g.key[0] == key || g.key[1] == key) return;  // already there or on its way
  fill_slot(h, 1 - g.last, nk, nset);
}

void residency_release(amg_hierarchy *h) {
  stager_free(h);
  for (auto &a : h->host_allocs) cudaFreeHost(a.first);
  h->host_allocs.clear();
  cudaGetLastError();
}

extern "C" amg_status amg_set_residency(amg_hierarchy *h, int residency, int first_level, amg_stream_t stream) {
  clear_stale_cuda_error();
  if (!h || residency < AMG_RESIDENT || residency > AMG_HOST_STAGED) return AMG_ERR_INVALID_ARG;
  if (residency != AMG_RESIDENT && (first_level < 0 || first_level >= h->L)) return AMG_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  // finish the hierarchy's earlier work before its arrays move
  AMG_CUDA(cudaStreamSynchronize(h->last_stream ? h->last_stream : h->stream));
  stager_free(h);
  reset_graphs(h);
  h->batch_desc_stale = 1;
  // back to device memory first, so that any change starts from one state
  AMG_TRY(move_levels(h, 0, false, false, s));
  h->residency = AMG_RESIDENT;
  h->res_first = 0;
  if (residency == AMG_RESIDENT) return AMG_OK;
  amg_status st = move_levels(h, first_level, true, residency == AMG_HOST_STAGED, s);
  if (st == AMG_OK) {
    h->residency = residency;
    h->res_first = first_level;
    if (residency == AMG_HOST_STAGED) st = stager_create(h);
  }
  if (st != AMG_OK) {
    stager_free(h);
    move_levels(h, 0, false, false, s);  // best effort: leave the hierarchy resident
    h->residency = AMG_RESIDENT;
    h->res_first = 0;
    return st;
  }
  // freed device blocks go back to the device, not only to the library's pool
  pool_trim();
  h->last_stream = s;
  return AMG_OK;
}

extern "C" amg_status amg_memory_info(const amg_hierarchy *h, uint64_t *device_bytes, uint64_t *host_bytes,
                                      uint64_t *staging_bytes, uint64_t *copied_bytes) {
  if (!h) return AMG_ERR_INVALID_ARG;
  uint64_t d = 0, hb = 0;
  for (const auto &a : h->allocs) d += a.second;
  for (const auto &a : h->host_allocs) hb += a.second;
  const uint64_t sb = h->stg ? 2ull * h->stg->slot_bytes : 0ull;
  if (device_bytes) *device_bytes = d + sb;
  if (host_bytes) *host_bytes = hb;
  if (staging_bytes) *staging_bytes = sb;
  if (copied_bytes) *copied_bytes = h->stg ? h->stg->copied : 0ull;
  return AMG_OK;
}
