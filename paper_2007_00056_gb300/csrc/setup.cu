// setup.cu -- device setup phase (Sec. 3 "setup phase"; coarsening Sec. 2.1).
//
// Per level: `passes` pairwise heavy-edge matchings, each run as synchronous
// rounds of mutual-heaviest-neighbour handshakes until a round pairs nothing
// (the fixed point equals the greedy edge-order matching of Algorithm 3 with
// ties broken toward the smaller index), aggregate ids by smallest member,
// and the Galerkin product A_c = P^T A P (Sec. 2.1.1) with a fixed summation
// order: coarse row I, its members ascending, each member row in stored order.
#include <algorithm>
#include <cmath>
#include <cstring>

#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

#define HEM_FREE (-2)

// ---------------------------------------------------------------------------
// CSR checks and diagonal
// ---------------------------------------------------------------------------
__global__ void k_check_csr(int n, long long nnz, const int32_t *__restrict__ rp,
                            const int32_t *__restrict__ ci, unsigned *eflags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && (rp[0] != 0 || (long long)rp[n] != nnz)) atomicOr(eflags, AMG_EFLAG_BAD_CSR);
  if (i >= n) return;
  int b = rp[i], e = rp[i + 1];
  if (b < 0 || e < b || (long long)e > nnz) { atomicOr(eflags, AMG_EFLAG_BAD_CSR); return; }
  int prev = -1;
  for (int k = b; k < e; ++k) {
    int c = ci[k];
    if (c < 0 || c >= n || c <= prev) { atomicOr(eflags, AMG_EFLAG_BAD_CSR); return; }
    prev = c;
  }
}

__device__ __forceinline__ int find_col(const int32_t *ci, int b, int e, int j) {
  int lo = b, hi = e - 1;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    int c = ci[mid];
    if (c == j) return mid;
    if (c < j) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

// dinv_i = 1 / a_ii; a missing, zero or non-finite diagonal sets a flag.
__global__ void k_diag(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                       const double *__restrict__ val, double *dinv, unsigned *eflags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int p = find_col(ci, rp[i], rp[i + 1], i);
  double d = p >= 0 ? val[p] : 0.0;
  if (d == 0.0 || !isfinite(d)) { atomicOr(eflags, AMG_EFLAG_ZERO_DIAG); dinv[i] = 0.0; return; }
  dinv[i] = 1.0 / d;
}

__global__ void k_nonfinite(long long nnz, const double *__restrict__ val, unsigned *eflags) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nnz;
       e += (long long)gridDim.x * blockDim.x)
    if (!isfinite(val[e])) { atomicOr(eflags, AMG_EFLAG_NONFINITE); return; }
}

// ---------------------------------------------------------------------------
// Edge weights: w_e = max(|a_ij|, |a_ji|) for e = (i, j), j != i; 0 = no edge.
// (Sec. 2.1: a_ij is the edge weight; Algorithm 3 lists both directions.)
// scaled != 0 (an option outside the paper): w_e / sqrt(|a_ii| * |a_jj|),
// which a zero diagonal turns into an error.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double abs_diag(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                           const double *__restrict__ val, int i) {
  const int p = find_col(ci, rp[i], rp[i + 1], i);
  return p >= 0 ? fabs(val[p]) : 0.0;
}

__global__ void k_weights(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                          const double *__restrict__ val, int scaled, double *__restrict__ w, unsigned *eflags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double di = scaled ? abs_diag(rp, ci, val, i) : 1.0;
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    int j = ci[e];
    if (j == i) { w[e] = 0.0; continue; }
    int q = find_col(ci, rp[j], rp[j + 1], i);
    double m;
    if (q < 0) {
      atomicOr(eflags, AMG_EFLAG_NONSYM);
      m = fabs(val[e]);
    } else {
      m = fmax(fabs(val[e]), fabs(val[q]));
    }
    if (scaled) {
      const double dd = di * abs_diag(rp, ci, val, j);
      if (!(dd > 0.0) || isinf(dd)) { atomicOr(eflags, AMG_EFLAG_ZERO_DIAG); m = 0.0; }
      else m = m / sqrt(dd);
    }
    w[e] = m;
  }
}

// ---------------------------------------------------------------------------
// Handshake rounds
// ---------------------------------------------------------------------------
__global__ void k_hem_init(int n, int32_t *mate, int32_t *dirty, int *stamp) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    mate[i] = HEM_FREE;
    dirty[i] = i;
    stamp[i] = 0;
  }
}

// Incremental rounds.  A free node's set of free neighbours only shrinks, so
// its pick (heaviest free neighbour, smaller index on equal weight) can change
// only when the node it picked was matched.  Round r therefore recomputes the
// picks of the nodes in its dirty list D_r only (D_0 = every node), pairs the
// mutual picks found from D_r, lists the newly matched nodes, and puts every
// free neighbour that had picked one of them into D_{r+1}.  The picks, pairs
// and round count equal those of recomputing every free node each round.
// Rounds run in batches between host checks: a round reads the sizes left by
// the previous round and does nothing once a previous round has paired
// nobody (the fixed point).  Lists are walked with grid-stride loops.
#define HEM_BLOCK_CAP 2048     // largest dirty list handled by the one-block rounds
#define HEM_BLOCK_ROUNDS 4096  // rounds per launch of the one-block rounds
#define HEM_COOP_THREADS 1024  // threads per block of the cooperative rounds (one block per SM)
// Counters of the cooperative rounds (ints), each on its own 128-byte line:
// the appended-list counters of three rounds (round r uses r % 3), the 64-bit
// barrier word, the result, and block 0's report after a solo stretch.
#define HEM_COOP_SLOT(r, f) (((r) % 3) * 64 + (f) * 32)  // f = 0: matched list M, 1: next list
#define HEM_COOP_BAR 192    // unsigned long long
#define HEM_COOP_OUT 224    // rounds run, finished
#define HEM_COOP_SOLO 256   // rounds, list size, finished, lists swapped
#define HEM_COOP_INTS 288
// Lists of at most HEM_SOLO_CAP nodes (one per thread of a block) run their
// rounds inside block 0 alone, through its L1 cache and block barriers, while
// the other blocks wait at a grid barrier: the narrow fronts of uniform grids
// and the last rounds of every pass.  At most HEM_SOLO_ROUNDS rounds per
// stretch keep every wait short.
#define HEM_SOLO_CAP HEM_COOP_THREADS
#define HEM_SOLO_ROUNDS 20000

// Slot for one appended list entry: the lanes of the warp that append at the
// same time share one atomic on the counter.
__device__ __forceinline__ int warp_append(int *counter) {
  cg::coalesced_group g = cg::coalesced_threads();
  int base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(counter, (int)g.size());
  return g.shfl(base, 0) + (int)g.thread_rank();
}

__device__ __forceinline__ int round_count(int n_host, const int *n_dev, const int *prev_matched) {
  if (prev_matched && *prev_matched == 0) return 0;
  return n_dev ? *n_dev : n_host;
}

// Picks of the dirty nodes; -1 when a node has no free neighbour left.
__global__ void k_hem_pick(int nd_host, const int *nd_dev, const int *prev_matched, const int32_t *__restrict__ D,
                           const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const double *__restrict__ w,
                           int tie_larger, const int32_t *__restrict__ mate, int32_t *__restrict__ pick) {
  const int nd = round_count(nd_host, nd_dev, prev_matched);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nd; t += gridDim.x * blockDim.x) {
    const int i = D[t];
    int best = -1;
    double bw = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      const double we = w[e];
      if (we <= 0.0) continue;
      const int j = ci[e];
      if (mate[j] != HEM_FREE) continue;
      // columns ascend, so on equal weight the first one met is the smaller
      // index and the last one the larger
      if (best < 0 || we > bw || (tie_larger && we == bw)) { best = j; bw = we; }
    }
    pick[i] = best;
  }
}

// Mutual picks seen from D_r become pairs (both ends written; the partner of a
// dirty node may be clean, its pick still valid).  Matched nodes are listed in
// M, each once: a partner that is itself dirty lists itself.  cnt[0] =
// matched nodes this round.
// Frontier rounds (full != 0) skip the dirty pass instead: D_r then holds
// every free node with a free neighbour (so both ends of a pair are in it),
// and D_{r+1} (cnt[1], stamp r + 1) is every node of D_r that picked but was
// not matched -- a superset of the dirty set, so incremental rounds may
// follow.  Cheaper than the dirty pass in the first rounds, where most pairs
// form; the host keeps them while a round pairs at least a sixteenth of its
// list and switches to incremental rounds for good after the first one that
// does not (a narrow front advancing through a uniform grid).
__global__ void k_hem_match(int nd_host, const int *nd_dev, const int *prev_matched, const int32_t *__restrict__ D,
                            int *__restrict__ stamp, int r, int full, const int32_t *__restrict__ pick,
                            int32_t *__restrict__ mate, int32_t *__restrict__ M, int32_t *__restrict__ Dn, int *cnt) {
  const int nd = round_count(nd_host, nd_dev, prev_matched);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nd; t += gridDim.x * blockDim.x) {
    const int i = D[t];
    const int j = pick[i];
    if (j < 0) continue;
    if (pick[j] != i) {
      if (full) {
        stamp[i] = r + 1;
        Dn[warp_append(&cnt[1])] = i;
      }
      continue;
    }
    mate[i] = j;
    if (full) {  // both ends are in D_r: each counts itself
      warp_append(&cnt[0]);
      continue;
    }
    mate[j] = i;
    M[warp_append(&cnt[0])] = i;
    if (stamp[j] != r) M[warp_append(&cnt[0])] = j;
  }
}

// D_{r+1}: free neighbours of this round's matched nodes whose pick was one of
// them, each listed once (stamp = r + 1).  cnt[1] = size of D_{r+1}.
__global__ void k_hem_dirty(const int *__restrict__ matched, const int32_t *__restrict__ M,
                            const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                            const int32_t *__restrict__ mate, const int32_t *__restrict__ pick, int *__restrict__ stamp,
                            int r1, int32_t *__restrict__ Dn, int *cnt) {
  const int nm = *matched;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nm; t += gridDim.x * blockDim.x) {
    const int m = M[t];
    for (int e = rp[m]; e < rp[m + 1]; ++e) {
      const int k = ci[e];
      if (k == m || mate[k] != HEM_FREE || pick[k] != m) continue;
      if (atomicExch(&stamp[k], r1) != r1) Dn[warp_append(&cnt[1])] = k;
    }
  }
}

// Incremental rounds while the dirty list is small run inside one thread block
// (the three steps of a round separated by block barriers, the list counters
// in shared memory): launches, not work, dominate such rounds on uniform
// grids, where thousands of them advance a narrow front.  The block leaves at
// the fixed point, when a next list exceeds `cap`, or after max_rounds.
// out[0] = rounds run (the last one pairing nobody counts), out[1] = 1 at the
// fixed point, out[2] = size of the list in D[out[3]].
__global__ void __launch_bounds__(1024)
    k_hem_rounds_block(int r0, int max_rounds, int cap, int nd, int32_t *__restrict__ Da, int32_t *__restrict__ Db,
                       int *__restrict__ stamp, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                       const double *__restrict__ w, int tie_larger, int32_t *__restrict__ mate,
                       int32_t *__restrict__ pick, int32_t *__restrict__ M, int *out) {
  __shared__ int s_nm, s_nn;
  int32_t *D = Da, *Dn = Db;
  int k = 0, finished = 0, which = 0;
  for (; k < max_rounds; ++k) {
    const int r = r0 + k;
    for (int t = threadIdx.x; t < nd; t += blockDim.x) {
      const int i = D[t];
      int best = -1;
      double bw = 0.0;
      for (int e = rp[i]; e < rp[i + 1]; ++e) {
        const double we = w[e];
        if (we <= 0.0) continue;
        const int j = ci[e];
        if (mate[j] != HEM_FREE) continue;
        if (best < 0 || we > bw || (tie_larger && we == bw)) { best = j; bw = we; }
      }
      pick[i] = best;
    }
    if (threadIdx.x == 0) {
      s_nm = 0;
      s_nn = 0;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nd; t += blockDim.x) {
      const int i = D[t];
      const int j = pick[i];
      if (j < 0 || pick[j] != i) continue;
      mate[i] = j;
      mate[j] = i;
      M[atomicAdd(&s_nm, 1)] = i;
      if (stamp[j] != r) M[atomicAdd(&s_nm, 1)] = j;
    }
    __syncthreads();
    const int nm = s_nm;
    if (nm == 0) {
      finished = 1;
      ++k;
      break;
    }
    for (int t = threadIdx.x; t < nm; t += blockDim.x) {
      const int m = M[t];
      for (int e = rp[m]; e < rp[m + 1]; ++e) {
        const int q = ci[e];
        if (q == m || mate[q] != HEM_FREE || pick[q] != m) continue;
        if (atomicExch(&stamp[q], r + 1) != r + 1) Dn[atomicAdd(&s_nn, 1)] = q;
      }
    }
    __syncthreads();
    nd = s_nn;
    int32_t *tmp = D;
    D = Dn;
    Dn = tmp;
    which ^= 1;
    __syncthreads();  // every thread has read s_nn before the next round resets it
    if (nd > cap) {
      ++k;
      break;
    }
  }
  if (threadIdx.x == 0) {
    out[0] = k;
    out[1] = finished;
    out[2] = nd;
    out[3] = which;
  }
}

// Heaviest free neighbour of i (smaller index on equal weight, or the larger
// one with tie_larger); -1 when i has no free neighbour.  mate is read past
// the L1 cache: other blocks of a persistent kernel write it.  The row is
// read eight entries at a time, all loads of a group issued before any is
// used, so a pick costs two dependent load latencies per group rather than
// two per entry; entries are still compared in stored (ascending) order.
#define HEM_GROUP 8
__device__ __forceinline__ int hem_pick_node(int i, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                             const double *__restrict__ w, int tie_larger, const int32_t *mate) {
  int best = -1;
  double bw = 0.0;
  const int e0 = __ldg(&rp[i]), e1 = __ldg(&rp[i + 1]);
  for (int base = e0; base < e1; base += HEM_GROUP) {
    int jj[HEM_GROUP], mm[HEM_GROUP];
    double ww[HEM_GROUP];
#pragma unroll
    for (int u = 0; u < HEM_GROUP; ++u) {
      const int e = base + u;
      jj[u] = e < e1 ? __ldg(&ci[e]) : -1;
      ww[u] = e < e1 ? __ldg(&w[e]) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < HEM_GROUP; ++u) mm[u] = (ww[u] > 0.0) ? __ldcg(&mate[jj[u]]) : 0;
#pragma unroll
    for (int u = 0; u < HEM_GROUP; ++u) {
      if (!(ww[u] > 0.0) || mm[u] != HEM_FREE) continue;
      if (best < 0 || ww[u] > bw || (tie_larger && ww[u] == bw)) { best = jj[u]; bw = ww[u]; }
    }
  }
  return best;
}

// Grid barrier whose 64-bit word also sums one value per block: the low half
// counts arrivals, the high half accumulates what each block adds on arrival,
// and the high half seen at completion is the total over every block up to
// this barrier (no block can add to the next barrier before all have passed
// this one).  Waits are bounded like GridBarrier's.
struct SumBarrier {
  unsigned long long *word;
  unsigned target;
  unsigned sleep_ns = 0;
  __device__ __forceinline__ bool sync(unsigned G, unsigned add, unsigned *eflags, int *fail_sh,
                                       unsigned *hi_sh, unsigned *hi_out) {
    __syncthreads();
    target += G;
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(word, 1ull | ((unsigned long long)add << 32));
      const long long t0 = clock64();
      unsigned long long v;
      for (;;) {
        asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(word) : "memory");
        if ((unsigned)v >= target) break;
        if (sleep_ns) __nanosleep(sleep_ns);
        if (clock64() - t0 > BARRIER_SPIN_LIMIT) {
          atomicOr(eflags, AMG_EFLAG_TIMEOUT);
          *fail_sh = 1;
          break;
        }
      }
      *hi_sh = (unsigned)(v >> 32);
    }
    __syncthreads();
    *hi_out = *hi_sh;
    return *fail_sh == 0;
  }
};

// Loads of the rounds' shared state: past L1 (other SMs write it) in grid
// rounds, through L1 inside a block's solo stretch.
template <bool L2ONLY>
__device__ __forceinline__ int ld_state(const int *p) { return L2ONLY ? __ldcg(p) : *p; }

// The graph of a matching pass as the rounds read it: CSR with edge weights,
// and, when every node has at most HEM_ELL neighbours, each node's neighbours
// sorted by preference (heaviest first, ties by the pass's index rule), -1
// padded: a pick is then the first free entry of one 32-byte row, with no
// weights and no row pointers on the round's dependent-load chain.
#define HEM_ELL 8
#define HEM_ELL_MIN_N 65536  // graphs up to this size skip the table
struct HemGraph {
  const int32_t *rp, *ci;
  const double *w;
  int tie_larger;
  const int32_t *nb;  // n x HEM_ELL sorted neighbours (ELL form only)
};

// Neighbours of u into jj[0..HEM_ELL) (-1 beyond the row) from the sorted
// table, two 16-byte loads.
__device__ __forceinline__ void hem_row_ell(const int32_t *__restrict__ nb, int u, int (&jj)[HEM_ELL]) {
  const int4 a = __ldg((const int4 *)(nb + (size_t)u * HEM_ELL));
  const int4 b = __ldg((const int4 *)(nb + (size_t)u * HEM_ELL) + 1);
  jj[0] = a.x; jj[1] = a.y; jj[2] = a.z; jj[3] = a.w;
  jj[4] = b.x; jj[5] = b.y; jj[6] = b.z; jj[7] = b.w;
}

// Heaviest free neighbour of q (the pass's tie rule), -1 when none.
template <bool L2ONLY, bool ELL>
__device__ __forceinline__ int hem_pick(int q, const HemGraph &g, const int32_t *mate) {
  if (ELL) {
    int jj[HEM_ELL], mm[HEM_ELL];
    hem_row_ell(g.nb, q, jj);
#pragma unroll
    for (int u = 0; u < HEM_ELL; ++u) mm[u] = jj[u] >= 0 ? ld_state<L2ONLY>(&mate[jj[u]]) : 0;
#pragma unroll
    for (int u = 0; u < HEM_ELL; ++u)
      if (mm[u] == HEM_FREE) return jj[u];
    return -1;
  }
  int best = -1;
  double bw = 0.0;
  const int e0 = __ldg(&g.rp[q]), e1 = __ldg(&g.rp[q + 1]);
  for (int base = e0; base < e1; base += HEM_GROUP) {
    int jj[HEM_GROUP], mm[HEM_GROUP];
    double ww[HEM_GROUP];
#pragma unroll
    for (int u = 0; u < HEM_GROUP; ++u) {
      const int e = base + u;
      jj[u] = e < e1 ? __ldg(&g.ci[e]) : -1;
      ww[u] = e < e1 ? __ldg(&g.w[e]) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < HEM_GROUP; ++u) mm[u] = (ww[u] > 0.0) ? ld_state<L2ONLY>(&mate[jj[u]]) : 0;
#pragma unroll
    for (int u = 0; u < HEM_GROUP; ++u) {
      if (!(ww[u] > 0.0) || mm[u] != HEM_FREE) continue;
      if (best < 0 || ww[u] > bw || (g.tie_larger && ww[u] == bw)) { best = jj[u]; bw = ww[u]; }
    }
  }
  return best;
}

// List appends staged in shared memory: a push takes a slot from a block
// counter; flush() reserves the block's range of the global list with one
// atomic and copies the staged entries out, so the global counter sees one
// atomic per block and flush instead of one per warp (thousands of atomics
// on one address serialise at its L2 slice).  Pushes beyond CAP between two
// flushes go straight to the global list.  Every thread of the block calls
// flush(); it returns the number of entries pushed since the last flush.
template <typename T, int CAP>
struct StagedList {
  T *buf;
  int *cnt, *base;
  T *out;
  int *gctr;
  __device__ __forceinline__ void push(T v) {
    const int k = atomicAdd(cnt, 1);
    if (k < CAP) buf[k] = v;
    else out[atomicAdd(gctr, 1)] = v;
  }
  __device__ __forceinline__ int flush() {
    __syncthreads();
    const int c = *cnt, m = c < CAP ? c : CAP;
    if (threadIdx.x == 0 && m) *base = atomicAdd(gctr, m);
    __syncthreads();
    const int b = *base;
    for (int k = threadIdx.x; k < m; k += blockDim.x) out[b + k] = buf[k];
    __syncthreads();
    if (threadIdx.x == 0) *cnt = 0;
    __syncthreads();
    return c;
  }
};
#define HEM_STAGE 3072  // staged entries per block between flushes

// Phase B, first half, for one newly matched node m of round r: every free
// neighbour q whose pick was m depends on m and must re-pick.  q is reached
// from m only (a node has one pick), so its stamp (r + 1: member of the next
// list) is a plain store.  Each dependant goes to `found`.
template <bool L2ONLY, bool ELL, typename FoundF>
__device__ __forceinline__ void hem_dependants(int m, int r, const HemGraph &g, const int32_t *mate,
                                               const int32_t *pick, int *stamp, FoundF found) {
  auto visit = [&](const int (&qq)[HEM_GROUP]) {
    int mq[HEM_GROUP], pq[HEM_GROUP];
#pragma unroll
    for (int u = 0; u < HEM_GROUP; ++u) {
      const bool other = qq[u] >= 0 && qq[u] != m;
      mq[u] = other ? ld_state<L2ONLY>(&mate[qq[u]]) : 0;
      pq[u] = other ? ld_state<L2ONLY>(&pick[qq[u]]) : -1;
    }
#pragma unroll
    for (int u = 0; u < HEM_GROUP; ++u) {
      const int q = qq[u];
      if (q < 0 || q == m || mq[u] != HEM_FREE || pq[u] != m) continue;
      stamp[q] = r + 1;
      found(q);
    }
  };
  if (ELL) {
    int qq[HEM_ELL];
    hem_row_ell(g.nb, m, qq);
    visit(qq);
    return;
  }
  const int e0 = __ldg(&g.rp[m]), e1 = __ldg(&g.rp[m + 1]);
  for (int base = e0; base < e1; base += HEM_GROUP) {
    int qq[HEM_GROUP];
#pragma unroll
    for (int u = 0; u < HEM_GROUP; ++u) qq[u] = base + u < e1 ? __ldg(&g.ci[base + u]) : -1;
    visit(qq);
  }
}

// Phase B of a block: the dependants of the matched nodes `nodes` (each
// thread passes the ones it holds; -1 for none) are collected in shared
// memory, then re-picked one per thread, so a thread's chain of dependent
// loads is one row scan and one pick rather than a scan and a pick per
// dependant.  Dependants beyond the shared list are re-picked where found.
// Every (q, new pick) goes to `emit`.  All threads of the block call it.
#define HEM_CAND 4096
template <bool L2ONLY, bool ELL, typename EmitF>
__device__ __forceinline__ void hem_phase_b(int m0, int m1, int r, const HemGraph &g, const int32_t *mate,
                                            int32_t *pick, int *stamp, int *cand, int *ncand, EmitF emit) {
  if (threadIdx.x == 0) *ncand = 0;
  __syncthreads();
  auto found = [&](int q) {
    const int k = atomicAdd(ncand, 1);
    if (k < HEM_CAND) {
      cand[k] = q;
    } else {
      const int np = hem_pick<L2ONLY, ELL>(q, g, mate);
      pick[q] = np;
      emit(make_int2(q, np));
    }
  };
  if (m0 >= 0) hem_dependants<L2ONLY, ELL>(m0, r, g, mate, pick, stamp, found);
  if (m1 >= 0) hem_dependants<L2ONLY, ELL>(m1, r, g, mate, pick, stamp, found);
  __syncthreads();
  const int nc = min(*ncand, HEM_CAND);
  for (int k = threadIdx.x; k < nc; k += blockDim.x) {
    const int q = cand[k];
    const int np = hem_pick<L2ONLY, ELL>(q, g, mate);
    pick[q] = np;
    emit(make_int2(q, np));
  }
}

// Sorted neighbour table of the ELL form: row i lists i's neighbours j with
// w_ij > 0, heaviest first, equal weights by the tie rule (smaller index
// first, or larger with tie_larger), -1 padded to HEM_ELL.  A row with more
// than HEM_ELL neighbours sets *too_wide (the pass then uses the CSR form).
__global__ void k_hem_ell(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                          const double *__restrict__ w, int tie_larger, int32_t *__restrict__ nb,
                          unsigned *too_wide) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int jj[HEM_ELL];
  double ww[HEM_ELL];
  int c = 0;
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    const double we = w[e];
    if (!(we > 0.0)) continue;
    if (c == HEM_ELL) { atomicOr(too_wide, 1u); return; }
    // insertion in preference order
    const int j = ci[e];
    int k = c++;
    while (k > 0 && (ww[k - 1] < we || (ww[k - 1] == we && (tie_larger ? jj[k - 1] < j : jj[k - 1] > j)))) {
      jj[k] = jj[k - 1];
      ww[k] = ww[k - 1];
      --k;
    }
    jj[k] = j;
    ww[k] = we;
  }
  for (int k = 0; k < HEM_ELL; ++k) nb[(size_t)i * HEM_ELL + k] = k < c ? jj[k] : -1;
}

// Every round of one matching pass in one cooperative launch (all blocks
// resident).  Round r, over the list D_r of (node, its pick):
//   A. each node i of D_r whose pick j picks i back is paired with j;
//   B. each newly matched node re-picks its dependants (hem_repick): free
//      neighbours whose pick it was, which form D_{r+1}.
// D_0 is every node (picks of phase 0, stamp 0).  Lists no longer than the
// grid's threads are handled one node per thread, the pair kept in registers
// across the barrier; longer ones go through the matched list M.  Lists of at
// most HEM_SOLO_CAP nodes run in block 0 alone (see HEM_SOLO_CAP).  The pass
// ends after the first round that pairs nobody; ctr[HEM_COOP_OUT] = rounds
// run (that last one included) and 1 when it ended (0: stopped at
// max_rounds or on a barrier timeout).  Picks, pairs and round counts are
// those of the synchronous rounds.
template <bool ELL>
__global__ void __launch_bounds__(HEM_COOP_THREADS)
    k_hem_coop(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const double *__restrict__ w,
               int tie_larger, const int32_t *__restrict__ nb, int32_t *mate, int32_t *pick, int *stamp, int2 *Da,
               int2 *Db, int32_t *M, int *ctr, unsigned *eflags, int max_rounds) {
  const HemGraph g{rp, ci, w, tie_larger, nb};
  __shared__ int fail_sh;
  __shared__ unsigned hi_sh;
  __shared__ int s_cnt, s_base, s_nc;
  __shared__ int2 s_d[HEM_STAGE];  // staged next-list entries (the matched list uses its first half as ints)
  __shared__ int s_c[HEM_CAND];    // dependants waiting for their new pick
  int *s_m = (int *)s_d;
  if (threadIdx.x == 0) { fail_sh = 0; s_cnt = 0; }
  const unsigned G = gridDim.x;
  SumBarrier gb{(unsigned long long *)(ctr + HEM_COOP_BAR), 0u};
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gstride = gridDim.x * blockDim.x;
  for (int i = gtid; i < n; i += gstride) pick[i] = hem_pick<true, ELL>(i, g, mate);
  unsigned hi = 0, hi_prev = 0;
  if (!gb.sync(G, 0, eflags, &fail_sh, &hi_sh, &hi)) return;
  hi_prev = hi;
  int2 *D = Da, *Dn = Db;
  int nd = n, r = 0;
  bool finished = false;
  while (r < max_rounds) {
    if (r > 0 && nd <= HEM_SOLO_CAP) {
      // short list: block 0 runs the next rounds alone, through its L1
      if (blockIdx.x == 0) {
        __shared__ int s_nn;
        asm volatile("fence.acq_rel.gpu;" ::: "memory");  // no stale L1 lines from before
        int2 *d = D, *dn = Dn;
        int lr = r, lnd = nd, fin = 0, swaps = 0;
        for (int k = 0; k < HEM_SOLO_ROUNDS && lr < max_rounds; ++k) {
          if (threadIdx.x == 0) s_nn = 0;
          __syncthreads();
          int mi = -1, mj = -1;
          if (threadIdx.x < lnd) {
            const int2 e = d[threadIdx.x];
            if (e.y >= 0 && pick[e.y] == e.x) {
              mate[e.x] = e.y;
              mate[e.y] = e.x;
              mi = e.x;
              mj = e.y;
            }
          }
          if (__syncthreads_or(mi >= 0) == 0) { fin = 1; ++lr; break; }
          auto app = [&](int2 v) { dn[atomicAdd(&s_nn, 1)] = v; };
          const int m1 = (mi >= 0 && stamp[mj] != lr) ? mj : -1;
          hem_phase_b<false, ELL>(mi, m1, lr, g, mate, pick, stamp, s_c, &s_nc, app);
          __syncthreads();
          lnd = s_nn;
          __syncthreads();  // every thread has read s_nn before the next round resets it
          int2 *tmp = d;
          d = dn;
          dn = tmp;
          swaps ^= 1;
          ++lr;
          if (lnd > HEM_SOLO_CAP) break;
        }
        if (threadIdx.x == 0) {
          ctr[HEM_COOP_SOLO + 0] = lr;
          ctr[HEM_COOP_SOLO + 1] = lnd;
          ctr[HEM_COOP_SOLO + 2] = fin;
          ctr[HEM_COOP_SOLO + 3] = swaps;
          for (int k = 0; k < 3; ++k) ctr[HEM_COOP_SLOT(k, 0)] = ctr[HEM_COOP_SLOT(k, 1)] = 0;
        }
      }
      gb.sleep_ns = 256;
      const bool ok = gb.sync(G, 0, eflags, &fail_sh, &hi_sh, &hi);
      gb.sleep_ns = 0;
      if (!ok) return;
      hi_prev = hi;
      r = __ldcg(&ctr[HEM_COOP_SOLO + 0]);
      nd = __ldcg(&ctr[HEM_COOP_SOLO + 1]);
      if (__ldcg(&ctr[HEM_COOP_SOLO + 3])) {
        int2 *tmp = D;
        D = Dn;
        Dn = tmp;
      }
      if (__ldcg(&ctr[HEM_COOP_SOLO + 2])) {
        finished = true;
        break;
      }
      continue;
    }
    int *cm = ctr + HEM_COOP_SLOT(r, 0), *cn = ctr + HEM_COOP_SLOT(r, 1);
    if (gtid == 0) {  // the counters of round r + 1 (last used by round r - 2)
      ctr[HEM_COOP_SLOT(r + 1, 0)] = 0;
      ctr[HEM_COOP_SLOT(r + 1, 1)] = 0;
    }
    // A: pairs.  One node per thread keeps its pair in registers; longer
    // lists list the matched nodes in M (each once)
    const bool regs = r > 0 && nd <= gstride;
    int mi = -1, mj = -1;
    bool any = false;
    if (regs) {
      if (gtid < nd) {
        const int2 e = __ldcg(&D[gtid]);
        if (e.y >= 0 && __ldcg(&pick[e.y]) == e.x) {
          mate[e.x] = e.y;
          mate[e.y] = e.x;
          mi = e.x;
          mj = e.y;
          any = true;
        }
      }
    } else {
      // chunks of one item per thread, the matched list staged per chunk
      StagedList<int, HEM_STAGE> ml{s_m, &s_cnt, &s_base, M, cm};
      for (int t0 = blockIdx.x * blockDim.x; t0 < nd; t0 += gstride) {
        const int t = t0 + threadIdx.x;
        if (t < nd) {
          int i, j;
          if (r == 0) { i = t; j = __ldcg(&pick[i]); }
          else { const int2 e = __ldcg(&D[t]); i = e.x; j = e.y; }
          if (j >= 0 && __ldcg(&pick[j]) == i) {
            mate[i] = j;
            mate[j] = i;
            any = true;
            ml.push(i);
            if (__ldcg(&stamp[j]) != r) ml.push(j);
          }
        }
        ml.flush();
      }
    }
    const int blk_any = __syncthreads_or(any);
    if (!gb.sync(G, blk_any ? 1u : 0u, eflags, &fail_sh, &hi_sh, &hi)) return;
    if (hi == hi_prev) {
      finished = true;
      ++r;
      break;
    }
    hi_prev = hi;
    // B: the next list, staged per block
    const int nm = regs ? 0 : __ldcg(cm);
    StagedList<int2, HEM_STAGE> nl{s_d, &s_cnt, &s_base, Dn, cn};
    auto app = [&](int2 v) { nl.push(v); };
    int added = 0;
    if (regs) {
      const int m1 = (mi >= 0 && __ldcg(&stamp[mj]) != r) ? mj : -1;
      hem_phase_b<true, ELL>(mi, m1, r, g, mate, pick, stamp, s_c, &s_nc, app);
      added = nl.flush();
    } else {
      for (int t0 = blockIdx.x * blockDim.x; t0 < nm; t0 += gstride) {
        const int t = t0 + threadIdx.x;
        hem_phase_b<true, ELL>(t < nm ? __ldcg(&M[t]) : -1, -1, r, g, mate, pick, stamp, s_c, &s_nc, app);
        added += nl.flush();
      }
    }
    if (!gb.sync(G, (unsigned)added, eflags, &fail_sh, &hi_sh, &hi)) return;
    nd = (int)(hi - hi_prev);
    hi_prev = hi;
    int2 *tmp = D;
    D = Dn;
    Dn = tmp;
    ++r;
  }
  if (gtid == 0) {
    ctr[HEM_COOP_OUT + 0] = r;
    ctr[HEM_COOP_OUT + 1] = finished ? 1 : 0;
  }
}

__global__ void k_hem_finish(int n, int32_t *mate) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && mate[i] == HEM_FREE) mate[i] = -1;
}

// ---------------------------------------------------------------------------
// Exclusive scan of int32 (three kernels: tile scan, scan of tile sums, add)
// ---------------------------------------------------------------------------
#define SCAN_ITEMS 8
#define SCAN_TILE (AMG_THREADS * SCAN_ITEMS)

__device__ __forceinline__ int block_excl_scan(int v, int *sh, int *total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int s = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    sh[lane] = s;  // inclusive over warps
  }
  __syncthreads();
  int warp_off = wid > 0 ? sh[wid - 1] : 0;
  *total = sh[(blockDim.x >> 5) - 1];
  __syncthreads();
  return warp_off + x - v;
}

__global__ void k_scan_tile(const int *in, int *out, int n, int *tile_sums) {
  __shared__ int sh[32];
  int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
  int v[SCAN_ITEMS];
  int s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    s += v[k];
  }
  int total;
  int off = block_excl_scan(s, sh, &total);
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    if (base + k < n) out[base + k] = off;
    off += v[k];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// One block: exclusive scan of the tile sums in chunks, carrying the running total.
__global__ void k_scan_sums(int *sums, int ntiles, int *total_out) {
  __shared__ int sh[32];
  int carry = 0;
  for (int base = 0; base < ntiles; base += blockDim.x) {
    int i = base + threadIdx.x;
    int v = i < ntiles ? sums[i] : 0;
    int tot;
    int ex = block_excl_scan(v, sh, &tot);
    if (i < ntiles) sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0 && total_out) *total_out = carry;
}

__global__ void k_scan_add(int *out, int n, const int *sums) {
  int base = blockIdx.x * SCAN_TILE;
  int add = sums[blockIdx.x];
  for (int k = threadIdx.x; k < SCAN_TILE; k += blockDim.x)
    if (base + k < n) out[base + k] += add;
}

// out[0..n-1] = exclusive scan of in, out[n] (if write_last) and *d_total = sum.
static void scan_excl(const int *in, int *out, int n, int *d_total, int *tiles, cudaStream_t s) {
  int nt = cdiv(std::max(n, 1), SCAN_TILE);
  k_scan_tile<<<nt, AMG_THREADS, 0, s>>>(in, out, n, tiles); count_launch();
  k_scan_sums<<<1, 1024, 0, s>>>(tiles, nt, d_total); count_launch();
  k_scan_add<<<nt, AMG_THREADS, 0, s>>>(out, n, tiles); count_launch();
}

// ---------------------------------------------------------------------------
// Aggregate numbering: id = rank of the aggregate's smallest member
// ---------------------------------------------------------------------------
__global__ void k_agg_flags(int n, const int32_t *__restrict__ mate, int *flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) { int m = mate[i]; flag[i] = (m < 0 || i < m) ? 1 : 0; }
}

__global__ void k_agg_assign(int n, const int32_t *__restrict__ mate, const int *__restrict__ id,
                             int32_t *__restrict__ agg, int32_t *__restrict__ first) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int m = mate[i];
  if (m < 0 || i < m) { agg[i] = id[i]; first[id[i]] = i; }
  else agg[i] = id[m];
}

// ---------------------------------------------------------------------------
// Galerkin product of one pairwise pass: coarse row I has members i0 = first[I]
// and i1 = mate[i0] (if paired, i1 > i0).  Its entries, in the order
// (row i0 in stored order, then row i1 in stored order), map to coarse columns
// J = agg[j]; distinct J are stored ascending, each value summed in that order
// starting from its first contribution.  One warp per coarse row.
// ---------------------------------------------------------------------------
struct PairRow {
  int b0, n0, b1, n1;
  __device__ __forceinline__ int m() const { return n0 + n1; }
  __device__ __forceinline__ int pos(int k) const { return k < n0 ? b0 + k : b1 + (k - n0); }
};

__device__ __forceinline__ PairRow pair_row(int I, const int32_t *first, const int32_t *mate, const int32_t *rp) {
  PairRow r;
  int i0 = first[I];
  int i1 = mate[i0];
  r.b0 = rp[i0];
  r.n0 = rp[i0 + 1] - r.b0;
  if (i1 > i0) { r.b1 = rp[i1]; r.n1 = rp[i1 + 1] - r.b1; }
  else { r.b1 = 0; r.n1 = 0; }
  return r;
}

// The product's operands gathered first, by independent threads: each coarse
// row's member row bounds (b0, n0, b1, n1) and each fine entry's coarse column
// agg[ci[e]].  The product then waits on two dependent loads per coarse row
// instead of five (first, mate, rp, ci, agg), which bound its time.
__global__ void k_pair_meta(int nc, const int32_t *__restrict__ first, const int32_t *__restrict__ mate,
                            const int32_t *__restrict__ rp, int4 *__restrict__ meta) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  const PairRow r = pair_row(I, first, mate, rp);
  meta[I] = make_int4(r.b0, r.n0, r.b1, r.n1);
}

__global__ void k_coarse_cols(long long nnz, const int32_t *__restrict__ ci, const int32_t *__restrict__ agg,
                              int32_t *__restrict__ Jf) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nnz; e += (long long)gridDim.x * blockDim.x)
    Jf[e] = agg[ci[e]];
}

#define GAL_WARPS (AMG_THREADS / 32)
#define GAL_CAP 256  // contributions per coarse row staged in shared memory

template <bool FILL>
__global__ void __launch_bounds__(AMG_THREADS)
    k_galerkin(int nc, const int4 *__restrict__ meta, const double *__restrict__ val, const int32_t *__restrict__ Jf,
               int *__restrict__ count, const int32_t *__restrict__ rpc, int32_t *__restrict__ cic,
               double *__restrict__ valc) {
  __shared__ int sJ[GAL_WARPS][GAL_CAP];
  __shared__ double sV[GAL_WARPS][GAL_CAP];
  __shared__ unsigned char sF[GAL_WARPS][GAL_CAP];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  // coarse rows in pairs: two rows of at most 16 contributions each take one
  // half-warp each (the same per-row steps and sum order as the full-warp
  // path below); any other row takes the whole warp
  for (int I2 = 2 * ((blockIdx.x * blockDim.x + threadIdx.x) >> 5); I2 < nc; I2 += 2 * warps) {
    const bool two = I2 + 1 < nc;
    const int4 mt0 = meta[I2];
    const int4 mt1 = two ? meta[I2 + 1] : make_int4(0, 0, 0, 0);
    if (two && mt0.y + mt0.w <= 16 && mt1.y + mt1.w <= 16) {
      const int h = lane >> 4, hl = lane & 15;
      const int4 mt = h ? mt1 : mt0;
      PairRow r;
      r.b0 = mt.x;
      r.n0 = mt.y;
      r.b1 = mt.z;
      r.n1 = mt.w;
      const int m = r.m();
      const int I = I2 + h;
      const int out0 = FILL ? rpc[I] : 0;
      const bool in = hl < m;
      const int J = in ? Jf[r.pos(hl)] : 0;
      const double v = in ? val[r.pos(hl)] : 0.0;
      // keys of the two halves never meet (bit 31 marks the second half,
      // coarse columns are below 2^31); unused lanes get distinct negatives
      const int key = in ? (int)((unsigned)J | ((unsigned)h << 31)) : -1 - lane;
      sV[wib][lane] = v;
      const unsigned grp = __match_any_sync(0xffffffffu, key);
      const bool firstJ = in && (grp & ((1u << lane) - 1u)) == 0u;
      __syncwarp();
      double sum = v;
      if (firstJ) {
        unsigned rest = grp & ~((2u << lane) - 1u);
        while (rest) {
          const int q = __ffs(rest) - 1;
          sum = __dadd_rn(sum, sV[wib][q]);
          rest &= rest - 1u;
        }
      }
      const unsigned fm = __ballot_sync(0xffffffffu, firstJ);
      int rank = 0;
      for (int k = 0; k < 16; ++k) {
        const int src = (h << 4) + k;
        const int Jk = __shfl_sync(0xffffffffu, J, src);
        if (k < m && ((fm >> src) & 1u) && Jk < J) ++rank;
      }
      if (FILL && firstJ) { cic[out0 + rank] = J; valc[out0 + rank] = sum; }
      if (!FILL && hl == 0) count[I] = __popc(fm & (h ? 0xffff0000u : 0x0000ffffu));
      __syncwarp();
      continue;
    }
    for (int u = 0; u < (two ? 2 : 1); ++u) {
    const int I = I2 + u;
    const int4 mt = u ? mt1 : mt0;
    PairRow r;
    r.b0 = mt.x;
    r.n0 = mt.y;
    r.b1 = mt.z;
    r.n1 = mt.w;
    const int m = r.m();
    int distinct = 0;
    const int out0 = FILL ? rpc[I] : 0;
    if (m <= 32) {
      // each lane holds one contribution (lanes >= m get distinct negative
      // keys); lanes with the same coarse column form a match group, the
      // group's lowest lane (first in stored order) sums its values in lane
      // order -- FP64 adds only for real duplicates
      const int J = lane < m ? Jf[r.pos(lane)] : -1 - lane;
      const double v = lane < m ? val[r.pos(lane)] : 0.0;
      sV[wib][lane] = v;
      const unsigned grp = __match_any_sync(0xffffffffu, J);
      const bool firstJ = lane < m && (grp & ((1u << lane) - 1u)) == 0u;
      __syncwarp();
      double sum = v;
      if (firstJ) {
        unsigned rest = grp & ~((2u << lane) - 1u);  // later lanes of the group, ascending
        while (rest) {
          const int q = __ffs(rest) - 1;
          sum = __dadd_rn(sum, sV[wib][q]);
          rest &= rest - 1u;
        }
      }
      const unsigned fm = __ballot_sync(0xffffffffu, firstJ);
      int rank = 0;
      for (int k = 0; k < m; ++k) {
        const int Jk = __shfl_sync(0xffffffffu, J, k);
        if (((fm >> k) & 1u) && Jk < J) ++rank;
      }
      distinct = __popc(fm);
      if (FILL && firstJ) { cic[out0 + rank] = J; valc[out0 + rank] = sum; }
      __syncwarp();
    } else if (m <= GAL_CAP) {
      // stage the contributions of this coarse row in the warp's shared slice
      int *J = sJ[wib];
      double *V = sV[wib];
      unsigned char *F = sF[wib];
      for (int k = lane; k < m; k += 32) { J[k] = Jf[r.pos(k)]; V[k] = val[r.pos(k)]; }
      __syncwarp();
      int cnt = 0;
      for (int k = lane; k < m; k += 32) {
        const int Jk = J[k];
        bool f = true;
        for (int q = 0; q < k; ++q)
          if (J[q] == Jk) { f = false; break; }
        F[k] = f ? 1 : 0;
        cnt += f ? 1 : 0;
      }
      __syncwarp();
      for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
      distinct = cnt;
      if (FILL) {
        for (int k = lane; k < m; k += 32) {
          if (!F[k]) continue;
          const int Jk = J[k];
          int rank = 0;
          double sum = V[k];
          for (int q = 0; q < m; ++q) {
            const int Jq = J[q];
            if (Jq < Jk && F[q]) ++rank;
            if (Jq == Jk && q > k) sum = __dadd_rn(sum, V[q]);
          }
          cic[out0 + rank] = Jk;
          valc[out0 + rank] = sum;
        }
      }
      __syncwarp();
    } else {
      // very long rows: the same definition with operands re-read from memory
      for (int k = lane; k < m; k += 32) {
        int J = Jf[r.pos(k)];
        bool firstJ = true;
        for (int q = 0; q < k && firstJ; ++q)
          if (Jf[r.pos(q)] == J) firstJ = false;
        if (!firstJ) continue;
        ++distinct;
        if (FILL) {
          int rank = 0;
          double sum = val[r.pos(k)];
          for (int q = 0; q < m; ++q) {
            int Jq = Jf[r.pos(q)];
            if (Jq < J) {
              bool fq = true;
              for (int u = 0; u < q && fq; ++u)
                if (Jf[r.pos(u)] == Jq) fq = false;
              if (fq) ++rank;
            } else if (Jq == J && q > k) {
              sum = __dadd_rn(sum, val[r.pos(q)]);
            }
          }
          cic[out0 + rank] = J;
          valc[out0 + rank] = sum;
        }
      }
      for (int o = 16; o > 0; o >>= 1) distinct += __shfl_xor_sync(0xffffffffu, distinct, o);
    }
    if (!FILL && lane == 0) count[I] = distinct;
    }
  }
}

// ---------------------------------------------------------------------------
// Composition of pass maps and member lists of the level's aggregates
// ---------------------------------------------------------------------------
__global__ void k_iota(int n, int32_t *a) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = i;
}
__global__ void k_compose(int n, int32_t *agg, const int32_t *__restrict__ pass_agg) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) agg[i] = pass_agg[agg[i]];
}
__global__ void k_count_members(int n, const int32_t *__restrict__ agg, int *cnt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(&cnt[agg[i]], 1);
}
__global__ void k_fill_members(int n, const int32_t *__restrict__ agg, const int32_t *__restrict__ mrp,
                               int *cursor, int32_t *mem) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int I = agg[i];
  int slot = atomicAdd(&cursor[I], 1);
  mem[mrp[I] + slot] = i;
}
// members ascending (insertion sort; aggregates hold at most 2^passes nodes)
__global__ void k_sort_members(int nc, const int32_t *__restrict__ mrp, int32_t *mem) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nc) return;
  int b = mrp[I], e = mrp[I + 1];
  for (int a = b + 1; a < e; ++a) {
    int v = mem[a], c = a - 1;
    while (c >= b && mem[c] > v) { mem[c + 1] = mem[c]; --c; }
    mem[c + 1] = v;
  }
}

// ---------------------------------------------------------------------------
// Residual-operator form of a zero-guess cycle visit (levels < L): the
// presmoothed iterate x = omega D^-1 f is folded into C = I - omega A D^-1,
// and prolongation plus postsmoothing into Q = P - omega D^-1 A P (see Level).
// One thread per row; setup only.
// ---------------------------------------------------------------------------
// c_ij = -a_ij (omega / a_jj) for j != i, c_ii = 1 - a_ii (omega / a_ii);
// wd_i = omega / a_ii.
__global__ void k_op_c(int n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                       const double *__restrict__ val, const double *__restrict__ dinv, double omega,
                       double *__restrict__ cval, double *__restrict__ wd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  wd[i] = omega * dinv[i];
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    const int j = ci[e];
    const double b = val[e] * (omega * dinv[j]);
    cval[e] = (j == i) ? 1.0 - b : -b;
  }
}

// Rows of up to OPQ_SHORT entries are handled by one thread (O(len^2) work on
// a handful of entries); longer rows (hub rows of stalled coarse levels) are
// handed to a whole warp, which stages the row's aggregate ids in shared
// memory (rows of up to OPQ_STAGE entries; longer ones read global memory)
// and marks in `first` the entries that are the first of their aggregate.
#define OPQ_SHORT 32
#define OPQ_STAGE 1024
#define OPQ_WARPS (AMG_THREADS / 32)

// Entries of row i of A P: the distinct aggregates agg[j] of its columns.
// Block: AMG_THREADS consecutive rows.
__global__ void __launch_bounds__(AMG_THREADS) k_op_qcount(int n, const int32_t *__restrict__ rp,
                                                           const int32_t *__restrict__ ci,
                                                           const int32_t *__restrict__ agg, int *__restrict__ cnt,
                                                           uint8_t *__restrict__ first) {
  __shared__ int longs[AMG_THREADS];
  __shared__ int nlong;
  __shared__ int stage[OPQ_WARPS][OPQ_STAGE];
  if (threadIdx.x == 0) nlong = 0;
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const int b = rp[i], e = rp[i + 1];
    if (e - b <= OPQ_SHORT) {
      int c = 0;
      for (int k = b; k < e; ++k) {
        const int a = agg[ci[k]];
        bool seen = false;
        for (int m = b; m < k && !seen; ++m) seen = agg[ci[m]] == a;
        c += seen ? 0 : 1;
      }
      cnt[i] = c;
    } else {
      longs[atomicAdd(&nlong, 1)] = i;
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int *sa = stage[w];
  for (int q = w; q < nlong; q += OPQ_WARPS) {
    const int r = longs[q], b = rp[r], len = rp[r + 1] - b;
    const bool staged = len <= OPQ_STAGE;
    if (staged)
      for (int k = lane; k < len; k += 32) sa[k] = agg[ci[b + k]];
    __syncwarp();
    int c = 0;
    for (int k = lane; k < len; k += 32) {
      const int a = staged ? sa[k] : agg[ci[b + k]];
      bool seen = false;
      for (int m = 0; m < k && !seen; ++m) seen = (staged ? sa[m] : agg[ci[b + m]]) == a;
      first[b + k] = seen ? 0 : 1;
      c += seen ? 0 : 1;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) cnt[r] = c;
    __syncwarp();
  }
}

// Row i of Q: columns J ascending; (A P)_iJ sums the row's a_ij with agg[j] = J
// in stored order (the first one starts the sum), and
// q_iJ = [J == agg[i]] - wd_i (A P)_iJ.  Same row split as k_op_qcount; in a
// long row, the lane holding the first entry of an aggregate computes its
// slot (the number of first entries with a smaller id) and its sum.
__global__ void __launch_bounds__(AMG_THREADS) k_op_qfill(int n, const int32_t *__restrict__ rp,
                                                          const int32_t *__restrict__ ci,
                                                          const double *__restrict__ val,
                                                          const int32_t *__restrict__ agg,
                                                          const double *__restrict__ wd,
                                                          const int32_t *__restrict__ qrp,
                                                          const uint8_t *__restrict__ first,
                                                          int32_t *__restrict__ qci, double *__restrict__ qval) {
  __shared__ int longs[AMG_THREADS];
  __shared__ int nlong;
  __shared__ int stage[OPQ_WARPS][OPQ_STAGE];
  if (threadIdx.x == 0) nlong = 0;
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const int b = rp[i], e = rp[i + 1];
    if (e - b <= OPQ_SHORT) {
      const int ai = agg[i];
      const double w = wd[i];
      int last = -1;
      for (int o = qrp[i]; o < qrp[i + 1]; ++o) {
        int J = 0x7fffffff;
        for (int k = b; k < e; ++k) {
          const int a = agg[ci[k]];
          if (a > last && a < J) J = a;
        }
        double sum = 0.0;
        bool fst = true;
        for (int k = b; k < e; ++k) {
          if (agg[ci[k]] != J) continue;
          sum = fst ? val[k] : sum + val[k];
          fst = false;
        }
        qci[o] = J;
        qval[o] = (J == ai ? 1.0 : 0.0) - w * sum;
        last = J;
      }
    } else {
      longs[atomicAdd(&nlong, 1)] = i;
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  int *sa = stage[wp];
  for (int q = wp; q < nlong; q += OPQ_WARPS) {
    const int r = longs[q], b = rp[r], len = rp[r + 1] - b, o0 = qrp[r], ar = agg[r];
    const double w = wd[r];
    const bool staged = len <= OPQ_STAGE;
    if (staged)
      for (int k = lane; k < len; k += 32) sa[k] = agg[ci[b + k]];
    __syncwarp();
    for (int k = lane; k < len; k += 32) {
      if (!first[b + k]) continue;
      const int a = staged ? sa[k] : agg[ci[b + k]];
      int slot = 0;
      for (int m = 0; m < len; ++m)
        if (first[b + m] && (staged ? sa[m] : agg[ci[b + m]]) < a) ++slot;
      double sum = val[b + k];
      for (int m = k + 1; m < len; ++m)
        if ((staged ? sa[m] : agg[ci[b + m]]) == a) sum = sum + val[b + m];
      qci[o0 + slot] = a;
      qval[o0 + slot] = (a == ar ? 1.0 : 0.0) - w * sum;
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

struct Scratch {
  double *w = nullptr;
  int32_t *mate = nullptr, *pick = nullptr, *fa = nullptr, *fb = nullptr, *first = nullptr;
  int *flag = nullptr, *id = nullptr, *tiles = nullptr, *cnt = nullptr, *count = nullptr;
  int *coop = nullptr;  // counters and barrier of the cooperative rounds (HEM_COOP_INTS)
  int2 *la = nullptr, *lb = nullptr;  // the cooperative rounds' lists of (node, pick)
  int32_t *nb = nullptr;              // sorted neighbour table (n x HEM_ELL)
  int *host = nullptr;  // pinned: [0] pairs, [1] frontier, [2] scan total
  size_t cap_n = 0, cap_nnz = 0;
};

struct Csr {
  int n = 0;
  long long nnz = 0;
  int32_t *rp = nullptr, *ci = nullptr;
  double *val = nullptr;
};

void free_csr(Csr &c, cudaStream_t st) {
  pool_free(c.rp, st); pool_free(c.ci, st); pool_free(c.val, st);
  c = Csr();
}

amg_status scratch_alloc(Scratch &s, int n, long long nnz, cudaStream_t st) {
  int tiles = cdiv(std::max(n, 1), SCAN_TILE);
  AMG_TRY(pool_alloc((void **)&s.w, sizeof(double) * (nnz + AMG_PAD), st));
  AMG_TRY(pool_alloc((void **)&s.mate, sizeof(int32_t) * (n + AMG_PAD), st));
  AMG_TRY(pool_alloc((void **)&s.pick, sizeof(int32_t) * (n + AMG_PAD), st));
  AMG_TRY(pool_alloc((void **)&s.fa, sizeof(int32_t) * (n + AMG_PAD), st));
  AMG_TRY(pool_alloc((void **)&s.fb, sizeof(int32_t) * (n + AMG_PAD), st));
  AMG_TRY(pool_alloc((void **)&s.first, sizeof(int32_t) * (n + AMG_PAD), st));
  AMG_TRY(pool_alloc((void **)&s.flag, sizeof(int) * (n + AMG_PAD), st));
  AMG_TRY(pool_alloc((void **)&s.id, sizeof(int) * (n + AMG_PAD), st));
  AMG_TRY(pool_alloc((void **)&s.count, sizeof(int) * (n + AMG_PAD), st));
  AMG_TRY(pool_alloc((void **)&s.tiles, sizeof(int) * (tiles + 8), st));
  AMG_TRY(pool_alloc((void **)&s.cnt, sizeof(int) * 64, st));
  AMG_TRY(pool_alloc((void **)&s.coop, sizeof(int) * HEM_COOP_INTS, st));
  AMG_TRY(pool_alloc((void **)&s.la, sizeof(int2) * (n + AMG_PAD), st));
  AMG_TRY(pool_alloc((void **)&s.lb, sizeof(int2) * (n + AMG_PAD), st));
  AMG_TRY(pool_alloc((void **)&s.nb, sizeof(int32_t) * ((size_t)n * HEM_ELL + AMG_PAD), st));
  s.host = (int *)pinned_small_alloc();
  if (!s.host) return AMG_ERR_OOM;
  s.cap_n = n;
  s.cap_nnz = nnz;
  return AMG_OK;
}

void scratch_free(Scratch &s, cudaStream_t st) {
  void *ps[] = {s.w, s.mate, s.pick, s.fa, s.fb, s.first, s.flag, s.id, s.count, s.tiles, s.cnt, s.coop, s.la, s.lb,
                s.nb};
  for (void *p : ps) pool_free(p, st);
  pinned_small_free(s.host);
  s = Scratch();
}

// Synchronous read of the device error bits (and reset).
amg_status check_flags(amg_hierarchy *h, cudaStream_t st) {
  unsigned f = 0;
  AMG_TRY(read_eflags(h, st, &f));
  if (f & AMG_EFLAG_BAD_CSR) return AMG_ERR_INVALID_CSR;
  if (f & AMG_EFLAG_NONFINITE) return AMG_ERR_INVALID_ARG;
  if (f & AMG_EFLAG_ZERO_DIAG) return AMG_ERR_ZERO_DIAG;
  if (f & AMG_EFLAG_NONSYM) return AMG_ERR_UNSUPPORTED;
  if (f & AMG_EFLAG_BREAKDOWN) return AMG_ERR_ZERO_DIAG;
  if (f & AMG_EFLAG_TIMEOUT) return AMG_ERR_TIMEOUT;
  return AMG_OK;
}

// Blocks of the cooperative handshake kernel on this device (one per SM), or
// 0 when the device cannot launch it cooperatively.
int hem_coop_blocks(amg_hierarchy *h, int n) {
  int coop = 0, occ = 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device) != cudaSuccess || !coop) {
    cudaGetLastError();
    return 0;
  }
  int occ2 = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_hem_coop<false>, HEM_COOP_THREADS, 0) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, k_hem_coop<true>, HEM_COOP_THREADS, 0) != cudaSuccess ||
      occ2 < 1 ||
      occ < 1) {
    cudaGetLastError();
    return 0;
  }
  // one block per 1024 nodes up to one per SM: a small graph's rounds take a
  // few blocks (a cheaper grid barrier) and leave the other SMs to the work
  // of other streams (measured: one block per 4096 nodes slowed the 128^3
  // lognormal setup from 14.1 to 17.2 ms, its coarse levels' wide rounds
  // wanting more blocks)
  return (int)std::min<long long>(h->num_sms, std::max<long long>(1, cdiv(n, 1024)));
}

// One pairwise pass on `in`: matching rounds, numbering, Galerkin product.
// pass_agg (n entries) receives the map; `out` the coarse CSR (allocated here).
amg_status coarsen_pass(amg_hierarchy *h, Scratch &S, const Csr &in, int32_t *pass_agg, Csr &out,
                        int *rounds, cudaStream_t st) {
  const int n = in.n;
  const int T = AMG_THREADS;
  const int tie_larger = h->prm.tie_break == AMG_TIE_LARGER ? 1 : 0;
  k_weights<<<cdiv(n, T), T, 0, st>>>(n, in.rp, in.ci, in.val, h->prm.edge_weight == AMG_WEIGHT_SCALED ? 1 : 0, S.w,
                                      h->eflags);
  count_launch();
  AMG_TRY(check_flags(h, st));
  // S.flag holds the round stamps and S.first the matched list while the
  // rounds run; the numbering below overwrites both
  k_hem_init<<<cdiv(n, T), T, 0, st>>>(n, S.mate, S.fa, S.flag); count_launch();
  int nd = n, r = 0;
  int32_t *fa = S.fa, *fb = S.fb;
  const int round_cap = 4 * n + 16;  // each productive round pairs >= 1 node
  int batch = 4;                     // rounds per host check: 4, 8, then 16
  bool finished = false, frontier_rounds = true;
  const int coop_blocks = hem_coop_blocks(h, n);
  bool coop_deferred = false;
  if (coop_blocks > 0) {
    // every round in one cooperative launch; the sorted neighbour table when
    // every node has at most HEM_ELL neighbours
    int *ctr = S.coop;
    AMG_CUDA(cudaMemsetAsync(ctr, 0, sizeof(int) * HEM_COOP_INTS, st));
    // the table pays on large graphs; a small one goes without it (and
    // without the host synchronisation that reads whether it fits)
    bool ell = false;
    if (n > HEM_ELL_MIN_N) {
      unsigned *too_wide = (unsigned *)(S.cnt + 60);
      AMG_CUDA(cudaMemsetAsync(too_wide, 0, sizeof(unsigned), st));
      k_hem_ell<<<cdiv(n, T), T, 0, st>>>(n, in.rp, in.ci, S.w, tie_larger, S.nb, too_wide);
      count_launch();
      AMG_CUDA(cudaMemcpyAsync(S.host + 60, too_wide, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
      AMG_CUDA(cudaStreamSynchronize(st));
      ell = S.host[60] == 0;
    }
    int a_n = n, a_tie = tie_larger, a_max = round_cap;
    const int32_t *a_rp = in.rp, *a_ci = in.ci;
    const double *a_w = S.w;
    int32_t *a_mate = S.mate, *a_pick = S.pick, *a_m = S.first;
    int2 *a_da = S.la, *a_db = S.lb;
    int *a_stamp = S.flag;
    const int32_t *a_nb = S.nb;
    unsigned *a_ef = h->eflags;
    void *args[] = {&a_n, &a_rp, &a_ci, &a_w, &a_tie, &a_nb, &a_mate, &a_pick, &a_stamp, &a_da, &a_db, &a_m,
                    &ctr, &a_ef, &a_max};
    AMG_CUDA(cudaLaunchCooperativeKernel(ell ? (void *)k_hem_coop<true> : (void *)k_hem_coop<false>, coop_blocks,
                                         HEM_COOP_THREADS, args, 0, st));
    count_launch();
    // the round count and the completion flag are read with the aggregate
    // count below (one synchronisation); the numbering kernels in between
    // only index by mate[], which holds node indices or -1 at any time
    AMG_CUDA(cudaMemcpyAsync(S.host + 44, ctr + HEM_COOP_OUT, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
    finished = true;
    coop_deferred = true;
  }
  const int grid = std::min(cdiv(std::max(n, 1), T), 8 * h->num_sms);
  while (!finished) {
    if (r > round_cap) return AMG_ERR_TIMEOUT;
    if (!frontier_rounds && nd <= HEM_BLOCK_CAP) {
      // small list: rounds inside one block until it grows or the matching ends
      k_hem_rounds_block<<<1, 1024, 0, st>>>(r, HEM_BLOCK_ROUNDS, HEM_BLOCK_CAP, nd, fa, fb, S.flag, in.rp, in.ci,
                                             S.w, tie_larger, S.mate, S.pick, S.first, S.cnt + 36);
      count_launch();
      AMG_CUDA(cudaMemcpyAsync(S.host, S.cnt + 36, sizeof(int) * 4, cudaMemcpyDeviceToHost, st));
      AMG_CUDA(cudaStreamSynchronize(st));
      r += S.host[0];
      finished = S.host[1] != 0;
      nd = S.host[2];
      if (S.host[3]) std::swap(fa, fb);
      continue;
    }
    AMG_CUDA(cudaMemsetAsync(S.cnt, 0, sizeof(int) * 2 * batch, st));
    int32_t *ba = fa, *bb = fb;
    for (int b = 0; b < batch; ++b) {
      const int *nd_dev = b ? S.cnt + 2 * (b - 1) + 1 : nullptr;
      const int *prev = b ? S.cnt + 2 * (b - 1) : nullptr;
      const int rr = r + b;
      k_hem_pick<<<grid, T, 0, st>>>(nd, nd_dev, prev, ba, in.rp, in.ci, S.w, tie_larger, S.mate, S.pick);
      count_launch();
      const int full = frontier_rounds ? 1 : 0;
      k_hem_match<<<grid, T, 0, st>>>(nd, nd_dev, prev, ba, S.flag, rr, full, S.pick, S.mate, S.first, bb,
                                       S.cnt + 2 * b);
      count_launch();
      if (!full) {
        k_hem_dirty<<<grid, T, 0, st>>>(S.cnt + 2 * b, S.first, in.rp, in.ci, S.mate, S.pick, S.flag, rr + 1, bb,
                                         S.cnt + 2 * b);
        count_launch();
      }
      std::swap(ba, bb);
    }
    AMG_CUDA(cudaMemcpyAsync(S.host, S.cnt, sizeof(int) * 2 * batch, cudaMemcpyDeviceToHost, st));
    AMG_CUDA(cudaStreamSynchronize(st));
    for (int b = 0; b < batch; ++b) {
      ++r;
      if (S.host[2 * b] == 0) { finished = true; break; }
      if (frontier_rounds && 16ll * S.host[2 * b] < (long long)nd) frontier_rounds = false;
      nd = S.host[2 * b + 1];
    }
    fa = ba;
    fb = bb;
    batch = std::min(batch * 2, 16);
  }
  *rounds = r;
  k_hem_finish<<<cdiv(n, T), T, 0, st>>>(n, S.mate); count_launch();
  // numbering
  k_agg_flags<<<cdiv(n, T), T, 0, st>>>(n, S.mate, S.flag); count_launch();
  scan_excl(S.flag, S.id, n, S.cnt + 34, S.tiles, st);
  k_agg_assign<<<cdiv(n, T), T, 0, st>>>(n, S.mate, S.id, pass_agg, S.first); count_launch();
  cudaMemcpyAsync(S.host + 34, S.cnt + 34, sizeof(int), cudaMemcpyDeviceToHost, st);
  AMG_CUDA(cudaStreamSynchronize(st));
  if (coop_deferred) {
    *rounds = S.host[44];
    if (!S.host[45]) {
      AMG_TRY(check_flags(h, st));
      return AMG_ERR_TIMEOUT;
    }
  }
  const int nc = S.host[34];
  // Galerkin: count, scan, fill
  out.n = nc;
  AMG_TRY(pool_alloc((void **)&out.rp, sizeof(int32_t) * (nc + 1 + AMG_PAD), st));
  const int gwarps_blocks = grid_for((long long)nc * 32, T, 152 * 16);
  // operands of the product (the matching's weight array and neighbour table
  // are free again): member row bounds and coarse columns of the fine entries
  int4 *meta = reinterpret_cast<int4 *>(S.nb);
  int32_t *Jf = reinterpret_cast<int32_t *>(S.w);
  k_pair_meta<<<cdiv(std::max(nc, 1), T), T, 0, st>>>(nc, S.first, S.mate, in.rp, meta); count_launch();
  k_coarse_cols<<<grid_for(std::max(in.nnz, 1ll), T, 152 * 16), T, 0, st>>>(in.nnz, in.ci, pass_agg, Jf);
  count_launch();
  k_galerkin<false><<<gwarps_blocks, T, 0, st>>>(nc, meta, in.val, Jf, S.count, nullptr, nullptr, nullptr);
  count_launch();
  scan_excl(S.count, out.rp, nc, S.cnt + 35, S.tiles, st);
  cudaMemcpyAsync(out.rp + nc, S.cnt + 35, sizeof(int), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(S.host + 35, S.cnt + 35, sizeof(int), cudaMemcpyDeviceToHost, st);
  AMG_CUDA(cudaStreamSynchronize(st));
  out.nnz = S.host[35];
  AMG_TRY(pool_alloc((void **)&out.ci, sizeof(int32_t) * (out.nnz + AMG_PAD), st));
  AMG_TRY(pool_alloc((void **)&out.val, sizeof(double) * (out.nnz + AMG_PAD), st));
  cudaMemsetAsync(out.ci + out.nnz, 0, sizeof(int32_t) * AMG_PAD, st);
  cudaMemsetAsync(out.val + out.nnz, 0, sizeof(double) * AMG_PAD, st);
  k_galerkin<true><<<gwarps_blocks, T, 0, st>>>(nc, meta, in.val, Jf, nullptr, out.rp, out.ci, out.val);
  count_launch();
  AMG_CUDA(cudaGetLastError());
  return AMG_OK;
}

amg_status validate_params(const amg_params *p) {
  if (p->passes < 1 || p->passes > AMG_MAX_PASSES) return AMG_ERR_INVALID_ARG;
  if (p->max_levels < 1 || p->max_levels > AMG_MAX_LEVELS) return AMG_ERR_INVALID_ARG;
  if (p->coarse_max < 1) return AMG_ERR_INVALID_ARG;
  if (!(p->stall_ratio > 0.0) || !(p->stall_ratio <= 1.0)) return AMG_ERR_INVALID_ARG;
  if (!(p->omega > 0.0) || !(p->omega < 2.0)) return AMG_ERR_INVALID_ARG;
  if (p->nu_pre < 1 || p->nu_post < 0 || p->nu_pre > 64 || p->nu_post > 64) return AMG_ERR_INVALID_ARG;
  if (p->coarse_solver < 0 || p->coarse_solver > 2) return AMG_ERR_INVALID_ARG;
  if (p->precision < 0 || p->precision > 2) return AMG_ERR_INVALID_ARG;
  if (p->cycle < AMG_CYCLE_V || p->cycle > AMG_CYCLE_F) return AMG_ERR_INVALID_ARG;
  if (p->tie_break != AMG_TIE_SMALLER && p->tie_break != AMG_TIE_LARGER) return AMG_ERR_INVALID_ARG;
  if (p->edge_weight != AMG_WEIGHT_ABS && p->edge_weight != AMG_WEIGHT_SCALED) return AMG_ERR_INVALID_ARG;
  if (p->operator_form != 0 && p->operator_form != 1) return AMG_ERR_INVALID_ARG;
  if (p->dense_max < 0) return AMG_ERR_INVALID_ARG;
  if (p->graphs < -1 || p->graphs > 1) return AMG_ERR_INVALID_ARG;
  return AMG_OK;
}

amg_status setup_impl(amg_hierarchy *h, int n, long long nnz, const int32_t *rp, const int32_t *ci,
                      const double *val, cudaStream_t st) {
  const int T = AMG_THREADS;
  // level 0: owned, padded copy of A
  Level &l0 = h->lev[0];
  l0.n = n;
  l0.nnz = nnz;
  AMG_TRY(hier_alloc(h, (void **)&l0.rp, sizeof(int32_t) * (n + 1 + AMG_PAD)));
  AMG_TRY(hier_alloc(h, (void **)&l0.ci, sizeof(int32_t) * (nnz + AMG_PAD)));
  AMG_TRY(hier_alloc(h, (void **)&l0.val, sizeof(double) * (nnz + AMG_PAD)));
  AMG_CUDA(cudaMemcpyAsync(l0.rp, rp, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToDevice, st));
  if (nnz) {
    AMG_CUDA(cudaMemcpyAsync(l0.ci, ci, sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice, st));
    AMG_CUDA(cudaMemcpyAsync(l0.val, val, sizeof(double) * nnz, cudaMemcpyDeviceToDevice, st));
  }
  cudaMemsetAsync(l0.ci + nnz, 0, sizeof(int32_t) * AMG_PAD, st);
  cudaMemsetAsync(l0.val + nnz, 0, sizeof(double) * AMG_PAD, st);
  k_check_csr<<<cdiv(n, T), T, 0, st>>>(n, nnz, l0.rp, l0.ci, h->eflags); count_launch();
  k_nonfinite<<<grid_for(nnz, T), T, 0, st>>>(nnz, l0.val, h->eflags); count_launch();
  AMG_TRY(check_flags(h, st));

  Scratch S;
  amg_status rs = scratch_alloc(S, n, nnz, st);
  if (rs != AMG_OK) { scratch_free(S, st); return rs; }
  int k = 0;
  const amg_params &p = h->prm;
  while (k + 1 < p.max_levels && h->lev[k].n > p.coarse_max) {
    Level &f = h->lev[k];
    Csr cur{f.n, f.nnz, f.rp, f.ci, f.val};
    bool owned = false;
    int32_t *agg = nullptr, *pass_agg = nullptr;
    rs = pool_alloc((void **)&agg, sizeof(int32_t) * (f.n + AMG_PAD), st);
    if (rs == AMG_OK) rs = pool_alloc((void **)&pass_agg, sizeof(int32_t) * (f.n + AMG_PAD), st);
    if (rs != AMG_OK) { pool_free(agg, st); scratch_free(S, st); return rs; }
    k_iota<<<cdiv(f.n, T), T, 0, st>>>(f.n, agg); count_launch();
    int rounds[AMG_MAX_PASSES] = {0};
    for (int pass = 0; pass < p.passes; ++pass) {
      Csr nxt;
      rs = coarsen_pass(h, S, cur, pass_agg, nxt, &rounds[pass], st);
      if (rs != AMG_OK) {
        free_csr(nxt, st);
        if (owned) free_csr(cur, st);
        pool_free(agg, st); pool_free(pass_agg, st); scratch_free(S, st);
        return rs;
      }
      k_compose<<<cdiv(f.n, T), T, 0, st>>>(f.n, agg, pass_agg); count_launch();
      if (owned) free_csr(cur, st);  // stream-ordered: after the kernels that read it
      cur = nxt;
      owned = true;
    }
    pool_free(pass_agg, st);
    if ((double)cur.n / (double)f.n > p.stall_ratio) {
      free_csr(cur, st);
      pool_free(agg, st);
      break;
    }
    // adopt the coarse level; record allocations for amg_destroy
    Level &c = h->lev[k + 1];
    c.n = cur.n;
    c.nnz = cur.nnz;
    c.rp = cur.rp; c.ci = cur.ci; c.val = cur.val;
    hier_adopt(h, cur.rp, sizeof(int32_t) * (cur.n + 1 + AMG_PAD));
    hier_adopt(h, cur.ci, sizeof(int32_t) * (cur.nnz + AMG_PAD));
    hier_adopt(h, cur.val, sizeof(double) * (cur.nnz + AMG_PAD));
    f.agg = agg;
    hier_adopt(h, agg, sizeof(int32_t) * (f.n + AMG_PAD));
    memcpy(f.rounds, rounds, sizeof(rounds));
    // member lists of the level's aggregates
    AMG_TRY(hier_alloc(h, (void **)&f.mrp, sizeof(int32_t) * (c.n + 1 + AMG_PAD)));
    AMG_TRY(hier_alloc(h, (void **)&f.mem, sizeof(int32_t) * (f.n + AMG_PAD)));
    cudaMemsetAsync(S.count, 0, sizeof(int) * c.n, st);
    k_count_members<<<cdiv(f.n, T), T, 0, st>>>(f.n, agg, S.count); count_launch();
    scan_excl(S.count, f.mrp, c.n, S.cnt + 36, S.tiles, st);
    cudaMemcpyAsync(f.mrp + c.n, S.cnt + 36, sizeof(int), cudaMemcpyDeviceToDevice, st);
    cudaMemsetAsync(S.count, 0, sizeof(int) * c.n, st);
    k_fill_members<<<cdiv(f.n, T), T, 0, st>>>(f.n, agg, f.mrp, S.count, f.mem); count_launch();
    k_sort_members<<<cdiv(c.n, T), T, 0, st>>>(c.n, f.mrp, f.mem); count_launch();
    AMG_CUDA(cudaGetLastError());
    ++k;
  }
  scratch_free(S, st);
  h->L = k;
  // diagonals of every level
  for (int j = 0; j <= h->L; ++j) {
    Level &l = h->lev[j];
    AMG_TRY(hier_alloc(h, (void **)&l.dinv, sizeof(double) * (l.n + AMG_PAD)));
    k_diag<<<cdiv(l.n, T), T, 0, st>>>(l.n, l.rp, l.ci, l.val, l.dinv, h->eflags); count_launch();
  }
  AMG_TRY(check_flags(h, st));
  return AMG_OK;
}

}  // namespace

// Forms C, Q and wd of every level below the coarsest (FP64; the FP32 mode's
// copies are made by precision_setup).  Only for one pre- and one post-sweep,
// and not in the FP16-storage mode, whose levels are scaled.
amg_status operator_form_setup(amg_hierarchy *h, cudaStream_t st) {
  const amg_params &p = h->prm;
  if (!p.operator_form || p.precision == AMG_FP16_STORAGE || p.nu_pre != 1 || p.nu_post != 1) return AMG_OK;
  const int T = AMG_THREADS;

  int nmax = 1;
  for (int k = 0; k < h->L; ++k) nmax = std::max(nmax, h->lev[k].n);
  long long nnzmax = 1;
  for (int k = 0; k < h->L; ++k) nnzmax = std::max(nnzmax, (long long)h->lev[k].nnz);
  int *cnt = nullptr, *tiles = nullptr, *tot = nullptr;
  uint8_t *first = nullptr;
  int *host = (int *)pinned_small_alloc();
  if (!host) return AMG_ERR_OOM;
  amg_status rs = pool_alloc((void **)&cnt, sizeof(int) * (nmax + AMG_PAD), st);
  if (rs == AMG_OK) rs = pool_alloc((void **)&tiles, sizeof(int) * (cdiv(nmax, SCAN_TILE) + 8), st);
  if (rs == AMG_OK) rs = pool_alloc((void **)&tot, sizeof(int) * 2 * AMG_MAX_LEVELS, st);
  if (rs == AMG_OK) rs = pool_alloc((void **)&first, (size_t)nnzmax + AMG_PAD, st);
  // level by level: the first-entry flags of a level are used by its fill
  for (int k = 0; k < h->L && rs == AMG_OK; ++k) {
    Level &l = h->lev[k];
    rs = hier_alloc(h, (void **)&l.cval, sizeof(double) * (l.nnz + AMG_PAD));
    if (rs == AMG_OK) rs = hier_alloc(h, (void **)&l.wd, sizeof(double) * (l.n + AMG_PAD));
    if (rs == AMG_OK) rs = hier_alloc(h, (void **)&l.qrp, sizeof(int32_t) * (l.n + 1 + AMG_PAD));
    if (rs != AMG_OK) break;
    cudaMemsetAsync(l.cval + l.nnz, 0, sizeof(double) * AMG_PAD, st);
    k_op_c<<<cdiv(l.n, T), T, 0, st>>>(l.n, l.rp, l.ci, l.val, l.dinv, p.omega, l.cval, l.wd); count_launch();
    k_op_qcount<<<cdiv(l.n, T), T, 0, st>>>(l.n, l.rp, l.ci, l.agg, cnt, first); count_launch();
    scan_excl(cnt, l.qrp, l.n, tot + k, tiles, st);
    cudaMemcpyAsync(l.qrp + l.n, tot + k, sizeof(int), cudaMemcpyDeviceToDevice, st);
    rs = amg_cuda_status(cudaMemcpyAsync(host, tot + k, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (rs == AMG_OK) rs = amg_cuda_status(cudaStreamSynchronize(st));
    if (rs != AMG_OK) break;
    l.qnnz = host[0];
    rs = hier_alloc(h, (void **)&l.qci, sizeof(int32_t) * (l.qnnz + AMG_PAD));
    if (rs == AMG_OK) rs = hier_alloc(h, (void **)&l.qval, sizeof(double) * (l.qnnz + AMG_PAD));
    if (rs != AMG_OK) break;
    cudaMemsetAsync(l.qci + l.qnnz, 0, sizeof(int32_t) * AMG_PAD, st);
    cudaMemsetAsync(l.qval + l.qnnz, 0, sizeof(double) * AMG_PAD, st);
    k_op_qfill<<<cdiv(l.n, T), T, 0, st>>>(l.n, l.rp, l.ci, l.val, l.agg, l.wd, l.qrp, first, l.qci, l.qval);
    count_launch();
    l.op_avail = 1;
    l.op_on = 1;
  }
  pinned_small_free(host);
  pool_free(cnt, st);
  pool_free(tiles, st);
  pool_free(tot, st);
  pool_free(first, st);
  if (rs != AMG_OK) return rs;
  return amg_cuda_status(cudaGetLastError());
}

extern "C" amg_status amg_setup(int n, int64_t nnz, const int32_t *d_row_ptr, const int32_t *d_col,
                                const double *d_val, const amg_params *params, amg_stream_t stream,
                                amg_hierarchy **out) {
  clear_stale_cuda_error();
  if (!out) return AMG_ERR_INVALID_ARG;
  *out = nullptr;
  if (n <= 0 || nnz < 0 || nnz >= (1ll << 31) - AMG_PAD || !d_row_ptr || (nnz > 0 && (!d_col || !d_val)))
    return AMG_ERR_INVALID_ARG;
  amg_params p;
  amg_default_params(&p);
  if (params) p = *params;
  AMG_TRY(validate_params(&p));
  cudaStream_t st = (cudaStream_t)stream;
  amg_hierarchy *h = new amg_hierarchy();
  h->prm = p;
  h->stream = st;
  h->last_stream = st;
  amg_status s = AMG_OK;
  do {
    if (cudaGetDevice(&h->device) != cudaSuccess) { s = AMG_ERR_CUDA; break; }
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) { s = AMG_ERR_CUDA; break; }
    s = hier_alloc(h, (void **)&h->eflags, sizeof(unsigned) * 4);
    if (s) break;
    h->eflags_host = (unsigned *)pinned_small_alloc();
    if (!h->eflags_host) { s = AMG_ERR_OOM; break; }
    cudaMemsetAsync(h->eflags, 0, sizeof(unsigned) * 4, st);
    s = setup_impl(h, n, nnz, d_row_ptr, d_col, d_val, st);
    if (s) break;
    s = coarse_setup(h, st);
    if (s) break;
    s = operator_form_setup(h, st);
    if (s) break;
    s = precision_setup(h, st);
    if (s) break;
    if (cudaStreamSynchronize(st) != cudaSuccess) { s = AMG_ERR_CUDA; break; }
  } while (0);
  if (s != AMG_OK) {
    cudaGetLastError();
    amg_destroy(h);
    return s;
  }
  *out = h;
  return AMG_OK;
}

extern "C" int amg_setup_rounds(const amg_hierarchy *h, int level, int pass) {
  if (!h || level < 0 || level >= h->L || pass < 0 || pass >= h->prm.passes) return -1;
  return h->lev[level].rounds[pass];
}
