// dense.cu -- dense inverse of the coarsest level, computed once at setup.
//
// The direct coarsest solve of Sec. 2 and Algorithm 1 ("solve exactly"),
// applied in every cycle as a matrix-vector product with A_L^-1.  The inverse
// comes from in-place Gauss-Jordan elimination with partial pivoting (pivot =
// the largest |entry| of the column at or below the diagonal, the smallest row
// index on ties), blocked by panels of nb columns:
//
//   1. one thread block factors the panel (all m rows x nb columns) in shared
//      memory, column by column: pivot search, row swap, scaling of the pivot
//      row, elimination of the column from every other row; in place, so the
//      panel ends up holding the panel's column of the elimination operator;
//   2. the panel's row swaps are applied to the other columns and the pivot
//      rows copied out (R, nb x m);
//   3. every other column is updated at once: M[i][j] = [i not a pivot row]
//      M[i][j] + sum_c panel[i][c] R[c][j], a rank-nb product;
//   4. after the last panel the columns are put back in order by undoing the
//      row interchanges in reverse.
//
// The elimination costs 2 m^3 flops.  This GPU issues FP64 at about 1/66 of
// its FP32 rate, so coarsest levels above GJ_FP64_MAX rows (where the FP64
// inverse would take over about 25 ms) are inverted in FP32 and each coarse
// solve refines in FP64 (r = f - A_L x, x += X r) a
// number of times fixed here at setup by measuring the convergence on a test
// vector: the fewest steps whose normwise backward error
// ||f - A x||_inf / (||A||_inf ||x||_inf + ||f||_inf) is at most GJ_BACKWARD_TOL,
// the accuracy of a backward-stable FP64 solve, plus one step of margin.  When
// the refinement does not get there the inverse is recomputed in FP64.
#include "common.cuh"

#define GJ_THREADS 1024
#define GJ_SMEM_MAX 231000       // dynamic shared memory of the panel kernel
#define GJ_FP64_MAX 2048         // largest coarsest level inverted in FP64 directly
#define GJ_TJ 256                // update kernel: columns per block (one per thread)
#define GJ_TI 32                 // update kernel: rows per block
#define GJ_REFINE_MAX 12         // refinement steps tried at setup
#define GJ_COLMAP_SMEM (4 * 32768)  // shared memory of k_gj_colmap (one int per column)
#define GJ_BACKWARD_TOL (16.0 * 2.220446049250313e-16)  // accepted backward error of the refined solve

namespace {

template <typename T>
__global__ void k_dense_zero(long long mm, T *__restrict__ M) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < mm; t += (long long)gridDim.x * blockDim.x)
    M[t] = (T)0;
}

// A (m x m CSR) into the dense row-major M with row stride ld >= m; rows and
// columns m..ld-1 (a padding) get the identity.
template <typename T>
__global__ void k_dense_scatter(int m, int ld, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                const double *__restrict__ val, T *__restrict__ M) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ld) return;
  if (i >= m) {
    M[(size_t)i * ld + i] = (T)1;
    return;
  }
  for (int e = rp[i]; e < rp[i + 1]; ++e) M[(size_t)i * ld + ci[e]] = (T)val[e];
}

// out (m x m) = the leading m x m block of W (row stride ld).
template <typename T>
__global__ void k_dense_crop(int m, int ld, const T *__restrict__ W, T *__restrict__ out) {
  const long long mm = (long long)m * m;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < mm; t += (long long)gridDim.x * blockDim.x)
    out[t] = W[(t / m) * ld + t % m];
}

// Step 1: factor columns k0 .. k0+nb-1 of the m x m array M in place (one
// block; the panel lives in shared memory with an odd row stride ldp).
template <typename T>
__global__ void __launch_bounds__(GJ_THREADS) k_gj_panel(int m, int k0, int nb, int ldp, T *__restrict__ M,
                                                         int *__restrict__ piv, unsigned *eflags) {
  extern __shared__ __align__(16) unsigned char gj_smem[];
  T *sp = (T *)gj_smem;
  __shared__ double wv[32];
  __shared__ int wi[32];
  __shared__ int p_sh, bad_sh;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  for (int idx = tid; idx < m * nb; idx += blockDim.x) {
    const int i = idx / nb, c = idx - i * nb;
    sp[i * ldp + c] = M[(size_t)i * m + k0 + c];
  }
  if (tid == 0) bad_sh = 0;
  __syncthreads();
  for (int c = 0; c < nb; ++c) {
    const int k = k0 + c;
    // pivot: largest |entry| in rows k.., smallest row on ties (each thread
    // visits its rows in ascending order, so a strict > keeps the first)
    double best = -1.0;
    int bi = m;
    for (int i = k + tid; i < m; i += blockDim.x) {
      const double a = fabs((double)sp[i * ldp + c]);
      if (a > best) {
        best = a;
        bi = i;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    if (lane == 0) {
      wv[wid] = best;
      wi[wid] = bi;
    }
    __syncthreads();
    if (wid == 0) {
      best = lane < nw ? wv[lane] : -1.0;
      bi = lane < nw ? wi[lane] : m;
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (lane == 0) {
        int p = bi;
        if (!(best > 0.0) || !isfinite(best) || p >= m) {
          bad_sh = 1;
          p = k;
        }
        p_sh = p;
        piv[k] = p;
      }
    }
    __syncthreads();
    const int p = p_sh;
    if (p != k) {
      for (int cc = tid; cc < nb; cc += blockDim.x) {
        const T t = sp[k * ldp + cc];
        sp[k * ldp + cc] = sp[p * ldp + cc];
        sp[p * ldp + cc] = t;
      }
    }
    __syncthreads();
    // scale the pivot row; in place, the pivot entry becomes 1/pivot
    const T pv = sp[k * ldp + c];
    const T d = pv != (T)0 ? (T)1 / pv : (T)0;
    __syncthreads();
    if (tid < nb) sp[k * ldp + tid] = (tid == c) ? d : sp[k * ldp + tid] * d;
    __syncthreads();
    // eliminate column c from every other row; in place, entry c becomes -f d
    const T *prow = sp + k * ldp;
    for (int i = tid; i < m; i += blockDim.x) {
      if (i == k) continue;
      T *row = sp + i * ldp;
      const T f = row[c];
      if (f != (T)0) {
        for (int cc = 0; cc < nb; ++cc) row[cc] = (cc == c ? (T)0 : row[cc]) - f * prow[cc];
      }
    }
    __syncthreads();
  }
  for (int idx = tid; idx < m * nb; idx += blockDim.x) {
    const int i = idx / nb, c = idx - i * nb;
    M[(size_t)i * m + k0 + c] = sp[i * ldp + c];
  }
  if (tid == 0 && bad_sh) atomicOr(eflags, AMG_EFLAG_BREAKDOWN);
}

// Step 2: the panel's row interchanges on every other column, in order, and
// the pivot rows copied to R (nb x m).  One thread per column.
template <typename T>
__global__ void k_gj_swap(int m, int k0, int nb, T *__restrict__ M, const int *__restrict__ piv, T *__restrict__ R) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m || (j >= k0 && j < k0 + nb)) return;
  for (int c = 0; c < nb; ++c) {
    const int k = k0 + c, p = piv[k];
    if (p != k) {
      const T t = M[(size_t)k * m + j];
      M[(size_t)k * m + j] = M[(size_t)p * m + j];
      M[(size_t)p * m + j] = t;
    }
  }
  for (int c = 0; c < nb; ++c) R[(size_t)c * m + j] = M[(size_t)(k0 + c) * m + j];
}

// Step 3: M[i][j] = [i not in the panel rows] M[i][j] + sum_c panel[i][c] R[c][j]
// for every column j outside the panel.  Block: GJ_TI rows x GJ_TJ columns;
// the panel rows of the tile in shared memory, a thread's column of R in
// registers.
template <typename T, int NB>
__global__ void __launch_bounds__(GJ_TJ) k_gj_update(int m, int k0, T *__restrict__ M, const T *__restrict__ R) {
  __shared__ T ps[GJ_TI][NB + 1];
  const int j = blockIdx.x * GJ_TJ + threadIdx.x;
  const int i0 = blockIdx.y * GJ_TI;
  for (int idx = threadIdx.x; idx < GJ_TI * NB; idx += GJ_TJ) {
    const int r = idx / NB, c = idx - r * NB, i = i0 + r;
    ps[r][c] = i < m ? M[(size_t)i * m + k0 + c] : (T)0;
  }
  __syncthreads();
  if (j >= m || (j >= k0 && j < k0 + NB)) return;
  T rr[NB];
#pragma unroll
  for (int c = 0; c < NB; ++c) rr[c] = R[(size_t)c * m + j];
  const int i1 = min(i0 + GJ_TI, m);
  for (int i = i0; i < i1; ++i) {
    T acc = (i >= k0 && i < k0 + NB) ? (T)0 : M[(size_t)i * m + j];
#pragma unroll
    for (int c = 0; c < NB; ++c) acc += ps[i - i0][c] * rr[c];
    M[(size_t)i * m + j] = acc;
  }
}

// Step 4: column map undoing the interchanges in reverse (one thread; the map
// lives in shared memory), then Out[i][j] = M[i][cm[j]].
__global__ void k_gj_colmap(int m, const int *__restrict__ piv, int *__restrict__ cm) {
  extern __shared__ int cm_sh[];
  if (threadIdx.x == 0) {
    for (int j = 0; j < m; ++j) cm_sh[j] = j;
    for (int k = m - 1; k >= 0; --k) {
      const int p = piv[k], t = cm_sh[k];
      cm_sh[k] = cm_sh[p];
      cm_sh[p] = t;
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < m; j += blockDim.x) cm[j] = cm_sh[j];
}

template <typename T>
__global__ void k_gj_unpermute(int m, const T *__restrict__ M, const int *__restrict__ cm, T *__restrict__ out) {
  const long long mm = (long long)m * m;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < mm; t += (long long)gridDim.x * blockDim.x) {
    const long long i = t / m;
    const int j = (int)(t - i * m);
    out[t] = M[i * m + cm[j]];
  }
}

template <typename T, int NB>
void gj_update_launch(int m, int k0, T *M, const T *R, cudaStream_t st) {
  dim3 grid(cdiv(m, GJ_TJ), cdiv(m, GJ_TI));
  k_gj_update<T, NB><<<grid, GJ_TJ, 0, st>>>(m, k0, M, R);
  count_launch();
}

// Panel widths with an instantiated update kernel.
template <typename T> struct GjWidths;
template <> struct GjWidths<float> {
  static constexpr int n = 9;
  static constexpr int w[9] = {32, 24, 16, 12, 8, 6, 4, 2, 1};
};
template <> struct GjWidths<double> {
  static constexpr int n = 5;
  static constexpr int w[5] = {8, 6, 4, 2, 1};
};

template <typename T>
void gj_update_dispatch(int nb, int m, int k0, T *M, const T *R, cudaStream_t st) {
  switch (nb) {
    case 32: gj_update_launch<T, 32>(m, k0, M, R, st); break;
    case 24: gj_update_launch<T, 24>(m, k0, M, R, st); break;
    case 16: gj_update_launch<T, 16>(m, k0, M, R, st); break;
    case 12: gj_update_launch<T, 12>(m, k0, M, R, st); break;
    case 8: gj_update_launch<T, 8>(m, k0, M, R, st); break;
    case 6: gj_update_launch<T, 6>(m, k0, M, R, st); break;
    case 4: gj_update_launch<T, 4>(m, k0, M, R, st); break;
    case 2: gj_update_launch<T, 2>(m, k0, M, R, st); break;
    default: gj_update_launch<T, 1>(m, k0, M, R, st); break;
  }
}

// Widest instantiated panel that fits shared memory (odd row stride).
template <typename T>
int gj_panel_width(int m, int *ldp_out) {
  const long long max_ldp = GJ_SMEM_MAX / ((long long)m * (long long)sizeof(T));
  for (int k = 0; k < GjWidths<T>::n; ++k) {
    const int nb = GjWidths<T>::w[k];
    const int ldp = nb | 1;
    if (ldp <= max_ldp && nb <= m) {
      *ldp_out = ldp;
      return nb;
    }
  }
  return 0;
}

// Blocked Gauss-Jordan inverse of the coarsest matrix into out (m x m, T).
template <typename T>
amg_status gj_inverse(amg_hierarchy *h, T *out, cudaStream_t st) {
  const Level &c = h->lev[h->L];
  const int m = c.n;
  int ldp = 0;
  const int nb = gj_panel_width<T>(m, &ldp);
  if (nb < 1) return AMG_ERR_UNSUPPORTED;
  const size_t smem = (size_t)m * ldp * sizeof(T);
  AMG_CUDA(cudaFuncSetAttribute(k_gj_panel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, GJ_SMEM_MAX));
  const long long mm = (long long)m * m;
  T *M = nullptr, *R = nullptr;
  int *piv = nullptr;
  if (pool_alloc((void **)&M, sizeof(T) * (size_t)mm, st) != AMG_OK) return AMG_ERR_OOM;
  if (pool_alloc((void **)&R, sizeof(T) * (size_t)nb * m + sizeof(int) * 2 * (size_t)(m + AMG_PAD), st) != AMG_OK) {
    pool_free(M, st);
    return AMG_ERR_OOM;
  }
  piv = (int *)(R + (size_t)nb * m);
  int *cm = piv + m + AMG_PAD;
  const int TB = AMG_THREADS;
  k_dense_zero<T><<<grid_for(mm, TB), TB, 0, st>>>(mm, M);
  count_launch();
  k_dense_scatter<T><<<cdiv(m, TB), TB, 0, st>>>(m, m, c.rp, c.ci, c.val, M);
  count_launch();
  for (int k0 = 0; k0 < m;) {
    // widest instantiated width within the panel width and the columns left
    int w = 1;
    for (int k = 0; k < GjWidths<T>::n; ++k)
      if (GjWidths<T>::w[k] <= nb && GjWidths<T>::w[k] <= m - k0) {
        w = GjWidths<T>::w[k];
        break;
      }
    k_gj_panel<T><<<1, GJ_THREADS, smem, st>>>(m, k0, w, ldp, M, piv, h->eflags);
    count_launch();
    if (w == m) break;  // a single panel covers the whole matrix
    k_gj_swap<T><<<cdiv(m, TB), TB, 0, st>>>(m, k0, w, M, piv, R);
    count_launch();
    gj_update_dispatch<T>(w, m, k0, M, R, st);
    k0 += w;
  }
  // a fixed limit for every m up to the largest dense level (32768 rows): the
  // attribute is process-wide, and a setup on another thread must not lower it
  // under this launch
  if (sizeof(int) * (size_t)m > GJ_COLMAP_SMEM) return AMG_ERR_UNSUPPORTED;
  AMG_CUDA(cudaFuncSetAttribute(k_gj_colmap, cudaFuncAttributeMaxDynamicSharedMemorySize, GJ_COLMAP_SMEM));
  k_gj_colmap<<<1, 256, sizeof(int) * m, st>>>(m, piv, cm);
  count_launch();
  k_gj_unpermute<T><<<grid_for(mm, TB), TB, 0, st>>>(m, M, cm, out);
  count_launch();
  pool_free(R, st);
  pool_free(M, st);
  return amg_cuda_status(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Blocked Gauss-Jordan inverse without row interchanges.  Block step K (BW
// columns, pivot block P = M_KK):
//   M_KJ <- P^-1 M_KJ,  M_IJ <- M_IJ - M_IK M_KJ (new),  M_IK <- -M_IK P^-1,
//   M_KK <- P^-1        (I, J outside K)
// after the last step M = A^-1.  Every step is a rank-BW product over the
// whole matrix, spread over the GPU, instead of BW sequential single-column
// eliminations in one thread block.  Without pivoting it is stable for the
// symmetric positive definite and diagonally dominant coarsest matrices of
// Galerkin hierarchies; any other matrix is caught either by a vanishing
// pivot (breakdown flag) or by the refinement test of dense_inverse, which
// then recomputes the inverse with partial pivoting.
// ---------------------------------------------------------------------------
#define BGJ_W 64  // block width

// Step 1: P^-1 of the w x w pivot block by unblocked Gauss-Jordan (one block
// of BGJ_W x 16 threads: thread (ty, tx) owns column tx of rows ty + 16 q).
template <typename T>
__global__ void __launch_bounds__(BGJ_W * 16) k_bgj_diag(int m, int k0, int w, const T *__restrict__ M,
                                                         T *__restrict__ Pinv, unsigned *eflags) {
  __shared__ T P[BGJ_W][BGJ_W + 1];
  const int tx = threadIdx.x & (BGJ_W - 1), ty = threadIdx.x / BGJ_W;
  for (int r = ty; r < w; r += 16) P[r][tx] = tx < w ? M[(size_t)(k0 + r) * m + k0 + tx] : (T)0;
  bool bad = false;
  __syncthreads();
  for (int c = 0; c < w; ++c) {
    const T pv = P[c][c];
    const bool ok = pv != (T)0 && isfinite((double)pv);
    bad |= !ok;
    const T d = ok ? (T)1 / pv : (T)0;
    // multipliers of this column, read before any thread changes them
    T f[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = ty + 16 * q;
      f[q] = r < w ? P[r][c] : (T)0;
    }
    __syncthreads();
    // pivot row scaled; its own entry becomes 1/pivot
    if (ty == 0 && tx < w) P[c][tx] = (tx == c) ? d : P[c][tx] * d;
    __syncthreads();
    // every other row: r_j -= f p_j (j != c); entry c becomes -f / pivot
    if (tx < w) {
      const T pc = P[c][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = ty + 16 * q;
        if (r >= w || r == c) continue;
        P[r][tx] = (tx == c) ? -f[q] * d : P[r][tx] - f[q] * pc;
      }
    }
    __syncthreads();
  }
  for (int r = ty; r < w; r += 16)
    if (tx < w) Pinv[r * w + tx] = P[r][tx];
  if (bad && threadIdx.x == 0) atomicOr(eflags, AMG_EFLAG_BREAKDOWN);
}

// Step 2: R = P^-1 M_K* for the columns outside K, stored in R (w x m) and in
// the K rows of M.  Block: BGJ_RC columns (all w rows; a block writes only the
// columns it read, so the update in place is safe); thread: one column, every
// 16th row.
// Shared memory of k_bgj_rows / k_bgj_cols: two BGJ_W x (BGJ_W + 1) tiles.
#define BGJ_TILE_SMEM(T) (2 * sizeof(T) * BGJ_W * (BGJ_W + 1))
// columns (rows) of M per block of k_bgj_rows (k_bgj_cols): 16 gives 4 x m / 64
// blocks, enough to cover the GPU at m = 4096 (64 blocks did not)
#define BGJ_RC 16

template <typename T>
__global__ void __launch_bounds__(256) k_bgj_rows(int m, int k0, int w, T *__restrict__ M, const T *__restrict__ Pinv,
                                                  T *__restrict__ R) {
  extern __shared__ __align__(16) unsigned char bgj_rs[];
  T(*Ps)[BGJ_W + 1] = (T(*)[BGJ_W + 1])bgj_rs;
  T(*Ms)[BGJ_W + 1] = Ps + BGJ_W;
  const int tid = threadIdx.x, j0 = blockIdx.x * BGJ_RC;
  for (int idx = tid; idx < w * w; idx += blockDim.x) Ps[idx / w][idx % w] = Pinv[idx];
  for (int idx = tid; idx < w * BGJ_RC; idx += blockDim.x) {
    const int r = idx / BGJ_RC, jj = idx % BGJ_RC, j = j0 + jj;
    Ms[r][jj] = j < m ? M[(size_t)(k0 + r) * m + j] : (T)0;
  }
  __syncthreads();
  const int jj = tid % BGJ_RC, j = j0 + jj, rg = tid / BGJ_RC;
  if (j >= m || (j >= k0 && j < k0 + w)) return;
  for (int r = rg; r < w; r += 256 / BGJ_RC) {
    T acc = (T)0;
    for (int c = 0; c < w; ++c) acc += Ps[r][c] * Ms[c][jj];
    R[(size_t)r * m + j] = acc;
    M[(size_t)(k0 + r) * m + j] = acc;
  }
}

// Step 3: M_IJ -= M_IK R_KJ for I, J outside K (old M_IK).  Tile BM x BN per
// block of 256 threads, TM x TN outputs per thread, both factors in shared
// memory.
template <typename T, int BM, int BN, int TM, int TN>
__global__ void __launch_bounds__(256) k_bgj_update(int m, int k0, int w, T *__restrict__ M, const T *__restrict__ R) {
  static_assert((BM / TM) * (BN / TN) == 256, "256 threads");
  extern __shared__ __align__(16) unsigned char bgj_smem[];
  T *As = (T *)bgj_smem;            // [w][BM]: M_IK transposed
  T *Bs = As + (size_t)BGJ_W * BM;  // [w][BN]: R_KJ
  const int tid = threadIdx.x;
  const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
  for (int idx = tid; idx < BM * w; idx += 256) {
    const int r = idx / w, c = idx - r * w, i = i0 + r;
    As[c * BM + r] = i < m ? M[(size_t)i * m + k0 + c] : (T)0;
  }
  for (int idx = tid; idx < w * BN; idx += 256) {
    const int c = idx / BN, jj = idx - c * BN, j = j0 + jj;
    Bs[c * BN + jj] = j < m ? R[(size_t)c * m + j] : (T)0;
  }
  __syncthreads();
  constexpr int NX = BN / TN, NY = BM / TM;
  const int tx = tid % NX, ty = tid / NX;
  T acc[TM][TN];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) acc[a][b] = (T)0;
  for (int c = 0; c < w; ++c) {
    T av[TM], bv[TN];
#pragma unroll
    for (int a = 0; a < TM; ++a) av[a] = As[c * BM + ty + a * NY];
#pragma unroll
    for (int b = 0; b < TN; ++b) bv[b] = Bs[c * BN + tx + b * NX];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TN; ++b) acc[a][b] += av[a] * bv[b];
  }
#pragma unroll
  for (int a = 0; a < TM; ++a) {
    const int i = i0 + ty + a * NY;
    if (i >= m || (i >= k0 && i < k0 + w)) continue;
#pragma unroll
    for (int b = 0; b < TN; ++b) {
      const int j = j0 + tx + b * NX;
      if (j >= m || (j >= k0 && j < k0 + w)) continue;
      T *p = M + (size_t)i * m + j;
      *p = *p - acc[a][b];
    }
  }
}

// Step 3 in FP32 for m a multiple of 4: the same products in the same order
// per entry (c = 0..w-1, one FMA each), with the operands read from shared
// memory four at a time.  Block: 128 x 128 outputs; thread (ty, tx) of 16 x 16
// owns rows {4 ty + a, 64 + 4 ty + a} and columns {4 tx + b, 64 + 4 tx + b}
// (a, b = 0..3), so each k step reads two float4 of M_IK and two of R_KJ for
// 64 FMAs.  Rows of the shared tiles are 132 floats apart: 16-byte aligned,
// and the transposing stores of M_IK (lanes on consecutive rows) hit distinct
// banks.
#define BGJ4_S 132
#define BGJ4_SMEM (2 * sizeof(float) * BGJ_W * BGJ4_S)

__global__ void __launch_bounds__(256) k_bgj_update4(int m, int k0, int w, float *__restrict__ M,
                                                     const float *__restrict__ R) {
  extern __shared__ __align__(16) unsigned char bgj4_smem[];
  float *As = (float *)bgj4_smem;     // [c][r]: M_IK transposed
  float *Bs = As + BGJ_W * BGJ4_S;    // [c][j]: R_KJ
  const int tid = threadIdx.x;
  const int i0 = blockIdx.y * 128, j0 = blockIdx.x * 128;
  const int wq = w >> 2;  // w is a multiple of 4 (k0 and m are)
  for (int idx = tid; idx < 128 * wq; idx += 256) {
    const int r = idx & 127, cq = idx >> 7, i = i0 + r;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < m) v = *reinterpret_cast<const float4 *>(M + (size_t)i * m + k0 + 4 * cq);
    As[(4 * cq + 0) * BGJ4_S + r] = v.x;
    As[(4 * cq + 1) * BGJ4_S + r] = v.y;
    As[(4 * cq + 2) * BGJ4_S + r] = v.z;
    As[(4 * cq + 3) * BGJ4_S + r] = v.w;
  }
  for (int idx = tid; idx < w * 32; idx += 256) {
    const int c = idx >> 5, jq = idx & 31, j = j0 + 4 * jq;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (j < m) v = *reinterpret_cast<const float4 *>(R + (size_t)c * m + j);
    *reinterpret_cast<float4 *>(Bs + c * BGJ4_S + 4 * jq) = v;
  }
  __syncthreads();
  const int tx = tid & 15, ty = tid >> 4;
  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
  for (int c = 0; c < w; ++c) {
    const float4 a0 = *reinterpret_cast<const float4 *>(As + c * BGJ4_S + 4 * ty);
    const float4 a1 = *reinterpret_cast<const float4 *>(As + c * BGJ4_S + 64 + 4 * ty);
    const float4 b0 = *reinterpret_cast<const float4 *>(Bs + c * BGJ4_S + 4 * tx);
    const float4 b1 = *reinterpret_cast<const float4 *>(Bs + c * BGJ4_S + 64 + 4 * tx);
    const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = __fmaf_rn(av[a], bv[b], acc[a][b]);
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int i = i0 + (a < 4 ? 4 * ty + a : 64 + 4 * ty + (a - 4));
    if (i >= m || (i >= k0 && i < k0 + w)) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = j0 + 64 * h + 4 * tx;  // four columns, all inside or all outside K
      if (j >= m || (j >= k0 && j < k0 + w)) continue;
      float4 *p = reinterpret_cast<float4 *>(M + (size_t)i * m + j);
      float4 v = *p;
      v.x = v.x - acc[a][4 * h + 0];
      v.y = v.y - acc[a][4 * h + 1];
      v.z = v.z - acc[a][4 * h + 2];
      v.w = v.w - acc[a][4 * h + 3];
      *p = v;
    }
  }
}

// Step 4: M_IK <- -M_IK P^-1 for I outside K, M_KK <- P^-1.  Block: BGJ_RC
// rows (all w columns, again only what it read); thread: one row, every 16th
// column.
template <typename T>
__global__ void __launch_bounds__(256) k_bgj_cols(int m, int k0, int w, T *__restrict__ M, const T *__restrict__ Pinv) {
  extern __shared__ __align__(16) unsigned char bgj_cs[];
  T(*Ps)[BGJ_W + 1] = (T(*)[BGJ_W + 1])bgj_cs;
  T(*Cs)[BGJ_W + 1] = Ps + BGJ_W;
  const int tid = threadIdx.x, i0 = blockIdx.x * BGJ_RC;
  for (int idx = tid; idx < w * w; idx += blockDim.x) Ps[idx / w][idx % w] = Pinv[idx];
  for (int idx = tid; idx < BGJ_RC * w; idx += blockDim.x) {
    const int r = idx / w, c = idx - r * w, i = i0 + r;
    Cs[r][c] = i < m ? M[(size_t)i * m + k0 + c] : (T)0;
  }
  __syncthreads();
  const int r = tid % BGJ_RC, cg = tid / BGJ_RC, i = i0 + r;
  if (i >= m) return;
  const bool in_k = i >= k0 && i < k0 + w;
  for (int c = cg; c < w; c += 256 / BGJ_RC) {
    T v;
    if (in_k) {
      v = Ps[i - k0][c];
    } else {
      T acc = (T)0;
      for (int q = 0; q < w; ++q) acc += Cs[r][q] * Ps[q][c];
      v = -acc;
    }
    M[(size_t)i * m + k0 + c] = v;
  }
}

template <typename T> struct BgjTile;
template <> struct BgjTile<float> { static constexpr int BM = 128, BN = 128, TM = 8, TN = 8; };
template <> struct BgjTile<double> { static constexpr int BM = 64, BN = 64, TM = 4, TN = 4; };

// Blocked Gauss-Jordan inverse without pivoting into out (m x m).  Returns
// AMG_ERR_BREAKDOWN when a pivot block step met a zero or non-finite pivot
// (out is then unusable).  Synchronises the stream.
template <typename T>
amg_status bgj_inverse(amg_hierarchy *h, T *out, cudaStream_t st) {
  using TL = BgjTile<T>;
  const Level &c = h->lev[h->L];
  const int n = c.n;
  // FP32: eliminate on an order rounded up to a multiple of 4 whose extra rows
  // and columns are an identity block (the inverse of diag(A, I) is
  // diag(A^-1, I), and the padding meets A's entries only through exact
  // zeros), so that every row is 16-byte aligned for the float4 update
  const int m = sizeof(T) == sizeof(float) ? (n + 3) / 4 * 4 : n;
  const long long mm = (long long)m * m;
  const size_t smem = sizeof(T) * (size_t)BGJ_W * (TL::BM + TL::BN);
  AMG_CUDA(cudaFuncSetAttribute(k_bgj_update<T, TL::BM, TL::BN, TL::TM, TL::TN>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const bool vec4 = sizeof(T) == sizeof(float);
  if (vec4)
    AMG_CUDA(cudaFuncSetAttribute(k_bgj_update4, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BGJ4_SMEM));
  const size_t tsmem = BGJ_TILE_SMEM(T);
  AMG_CUDA(cudaFuncSetAttribute(k_bgj_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsmem));
  AMG_CUDA(cudaFuncSetAttribute(k_bgj_cols<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tsmem));
  T *R = nullptr;
  if (pool_alloc((void **)&R, sizeof(T) * ((size_t)BGJ_W * m + (size_t)BGJ_W * BGJ_W), st) != AMG_OK)
    return AMG_ERR_OOM;
  T *Pinv = R + (size_t)BGJ_W * m;
  T *const dst = out;
  if (m != n && pool_alloc((void **)&out, sizeof(T) * (size_t)mm, st) != AMG_OK) {
    pool_free(R, st);
    return AMG_ERR_OOM;
  }
  const int TB = AMG_THREADS;
  k_dense_zero<T><<<grid_for(mm, TB), TB, 0, st>>>(mm, out);
  k_dense_scatter<T><<<cdiv(m, TB), TB, 0, st>>>(n, m, c.rp, c.ci, c.val, out);
  count_launch(2);
  const dim3 ug(cdiv(m, TL::BN), cdiv(m, TL::BM));
  for (int k0 = 0; k0 < m; k0 += BGJ_W) {
    const int w = std::min(BGJ_W, m - k0);
    k_bgj_diag<T><<<1, BGJ_W * 16, 0, st>>>(m, k0, w, out, Pinv, h->eflags);
    k_bgj_rows<T><<<cdiv(m, BGJ_RC), 256, tsmem, st>>>(m, k0, w, out, Pinv, R);
    if (vec4)
      k_bgj_update4<<<ug, 256, BGJ4_SMEM, st>>>(m, k0, w, (float *)out, (const float *)R);
    else
      k_bgj_update<T, TL::BM, TL::BN, TL::TM, TL::TN><<<ug, 256, smem, st>>>(m, k0, w, out, R);
    k_bgj_cols<T><<<cdiv(m, BGJ_RC), 256, tsmem, st>>>(m, k0, w, out, Pinv);
    count_launch(4);
  }
  if (m != n) {
    k_dense_crop<T><<<grid_for((long long)n * n, TB), TB, 0, st>>>(n, m, out, dst);
    count_launch();
    pool_free(out, st);
  }
  AMG_CUDA(cudaGetLastError());
  unsigned flags = 0;
  amg_status rs = read_eflags(h, st, &flags);
  pool_free(R, st);
  AMG_TRY(rs);
  const unsigned others = flags & ~AMG_EFLAG_BREAKDOWN;
  if (others) {  // not ours: leave them for the caller's next check
    h->eflags_host[0] = others;
    AMG_CUDA(cudaMemcpyAsync(h->eflags, h->eflags_host, sizeof(unsigned), cudaMemcpyHostToDevice, st));
    AMG_CUDA(cudaStreamSynchronize(st));
  }
  if (flags & AMG_EFLAG_BREAKDOWN) return AMG_ERR_BREAKDOWN;
  return AMG_OK;
}

// Refinement test vector: f = A_L v for v_i = 1 + (i mod 7)/8.
__global__ void k_refine_rhs(int m, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                             const double *__restrict__ val, double *__restrict__ f) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double s = 0.0;
  for (int e = rp[i]; e < rp[i + 1]; ++e) s += val[e] * (1.0 + (double)(ci[e] % 7) / 8.0);
  f[i] = s;
}

}  // namespace

namespace {

// x = X f with the FP64 inverse (warp per row), for the accuracy check of an
// inverse formed without pivoting.
__global__ void k_gemv64_check(int m, const double *__restrict__ X, const double *__restrict__ f,
                               double *__restrict__ x) {
  const int lane = threadIdx.x & 31;
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= m) return;
  double s = 0.0;
  for (int j = lane; j < m; j += 32) s += X[(size_t)row * m + j] * f[j];
  s = warp_sum(s);
  if (lane == 0) x[row] = s;
}

// Whether the FP64 inverse in h->ainv solves a test system to the backward
// error of a stable FP64 solve (x = X f, no refinement).
amg_status inverse64_ok(amg_hierarchy *h, cudaStream_t st, bool *ok) {
  const Level &c = h->lev[h->L];
  const int m = c.n;
  *ok = false;
  double *f = nullptr;
  if (pool_alloc((void **)&f, sizeof(double) * 2 * ((size_t)m + AMG_PAD), st) != AMG_OK) return AMG_ERR_OOM;
  double *x = f + (m + AMG_PAD);
  const int TB = AMG_THREADS;
  k_refine_rhs<<<cdiv(m, TB), TB, 0, st>>>(m, c.rp, c.ci, c.val, f);
  k_gemv64_check<<<cdiv((long long)m * 32, TB), TB, 0, st>>>(m, h->ainv, f, x);
  count_launch(2);
  const long long nnz = c.nnz;
  std::vector<int32_t> hrp(m + 1), hci(nnz);
  std::vector<double> hval(nnz), hf(m), hx(m);
  cudaError_t ce = cudaMemcpyAsync(hrp.data(), c.rp, sizeof(int32_t) * (m + 1), cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess && nnz)
    ce = cudaMemcpyAsync(hci.data(), c.ci, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess && nnz)
    ce = cudaMemcpyAsync(hval.data(), c.val, sizeof(double) * nnz, cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(hf.data(), f, sizeof(double) * m, cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(hx.data(), x, sizeof(double) * m, cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  pool_free(f, st);
  if (ce != cudaSuccess) return amg_cuda_status(ce);
  double norm_a = 0.0, norm_f = 0.0, norm_x = 0.0, res = 0.0;
  bool finite = true;
  for (int i = 0; i < m; ++i) {
    double rs = 0.0, ax = 0.0;
    for (int e = hrp[i]; e < hrp[i + 1]; ++e) {
      rs += std::fabs(hval[e]);
      ax += hval[e] * hx[hci[e]];
    }
    norm_a = std::max(norm_a, rs);
    norm_f = std::max(norm_f, std::fabs(hf[i]));
    norm_x = std::max(norm_x, std::fabs(hx[i]));
    res = std::max(res, std::fabs(hf[i] - ax));
    if (!std::isfinite(hx[i])) finite = false;
  }
  *ok = finite && res <= GJ_BACKWARD_TOL * (norm_a * norm_x + norm_f);
  return AMG_OK;
}

// Refinement steps the FP32 inverse in h->ainv32 needs: the fewest steps s
// whose refined solve of a test system has a normwise backward error of at
// most GJ_BACKWARD_TOL, plus one step of margin; -1 when no s <= GJ_REFINE_MAX
// gets there.
amg_status refine_steps(amg_hierarchy *h, cudaStream_t st, int *steps_out) {
  const Level &c = h->lev[h->L];
  const int m = c.n;
  *steps_out = -1;
  double *f = nullptr;
  if (pool_alloc((void **)&f, sizeof(double) * 2 * ((size_t)m + AMG_PAD), st) != AMG_OK) return AMG_ERR_OOM;
  double *x = f + (m + AMG_PAD);
  const int TB = AMG_THREADS;
  k_refine_rhs<<<cdiv(m, TB), TB, 0, st>>>(m, c.rp, c.ci, c.val, f);
  count_launch();
  // the coarsest matrix and f on the host, for the backward error of each trial
  const long long nnz = c.nnz;
  std::vector<int32_t> hrp(m + 1), hci(nnz);
  std::vector<double> hval(nnz), hf(m), hx(m);
  cudaError_t ce = cudaMemcpyAsync(hrp.data(), c.rp, sizeof(int32_t) * (m + 1), cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess && nnz)
    ce = cudaMemcpyAsync(hci.data(), c.ci, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess && nnz)
    ce = cudaMemcpyAsync(hval.data(), c.val, sizeof(double) * nnz, cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(hf.data(), f, sizeof(double) * m, cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) {
    pool_free(f, st);
    return amg_cuda_status(ce);
  }
  double norm_a = 0.0, norm_f = 0.0;
  for (int i = 0; i < m; ++i) {
    double rs = 0.0;
    for (int e = hrp[i]; e < hrp[i + 1]; ++e) rs += std::fabs(hval[e]);
    norm_a = std::max(norm_a, rs);
    norm_f = std::max(norm_f, std::fabs(hf[i]));
  }
  for (int s = 0; s <= GJ_REFINE_MAX; ++s) {
    amg_status rs = dense_refined_solve<double>(h, f, x, s, st, nullptr);
    if (rs == AMG_OK && cudaMemcpyAsync(hx.data(), x, sizeof(double) * m, cudaMemcpyDeviceToHost, st) != cudaSuccess)
      rs = AMG_ERR_CUDA;
    if (rs == AMG_OK && cudaStreamSynchronize(st) != cudaSuccess) rs = AMG_ERR_CUDA;
    if (rs != AMG_OK) {
      pool_free(f, st);
      return rs;
    }
    double res = 0.0, norm_x = 0.0;
    bool finite = true;
    for (int i = 0; i < m; ++i) {
      if (!std::isfinite(hx[i])) finite = false;
      norm_x = std::max(norm_x, std::fabs(hx[i]));
      double ax = 0.0;
      for (int e = hrp[i]; e < hrp[i + 1]; ++e) ax += hval[e] * hx[hci[e]];
      res = std::max(res, std::fabs(hf[i] - ax));
    }
    if (!finite) break;
    if (res <= GJ_BACKWARD_TOL * (norm_a * norm_x + norm_f)) {
      *steps_out = s + 1;  // one step of margin
      break;
    }
  }
  pool_free(f, st);
  return AMG_OK;
}

}  // namespace

amg_status dense_inverse(amg_hierarchy *h, cudaStream_t st) {
  const Level &c = h->lev[h->L];
  const int m = c.n;
  h->ainv = nullptr;
  h->ainv32 = nullptr;
  h->dense_refine = 0;
  if (m > GJ_FP64_MAX) {
    AMG_TRY(hier_alloc(h, (void **)&h->ainv32, sizeof(float) * ((size_t)m * m + AMG_PAD)));
    AMG_TRY(hier_alloc(h, (void **)&h->dense_r, sizeof(double) * 2 * ((size_t)m + AMG_PAD)));
    // FP32 inverse: first without row interchanges (blocked over the whole
    // GPU), then, if a pivot vanished or the refinement does not reach FP64
    // accuracy, with partial pivoting
    for (int pivoting = 0; pivoting < 2; ++pivoting) {
      if (!pivoting) {
        amg_status rs = bgj_inverse<float>(h, h->ainv32, st);
        if (rs == AMG_ERR_BREAKDOWN) continue;
        AMG_TRY(rs);
      } else {
        AMG_TRY(gj_inverse<float>(h, h->ainv32, st));
      }
      int steps = -1;
      AMG_TRY(refine_steps(h, st, &steps));
      if (steps >= 0) {
        h->dense_refine = steps;
        return AMG_OK;
      }
    }
    h->ainv32 = nullptr;  // refinement does not reach FP64 accuracy: FP64 inverse
  }
  AMG_TRY(hier_alloc(h, (void **)&h->ainv, sizeof(double) * ((size_t)m * m + AMG_PAD)));
  // FP64 inverse: without row interchanges if that is accurate, else pivoted
  if (m > BGJ_W) {
    amg_status rs = bgj_inverse<double>(h, h->ainv, st);
    if (rs != AMG_ERR_BREAKDOWN) {
      AMG_TRY(rs);
      bool ok = false;
      AMG_TRY(inverse64_ok(h, st, &ok));
      if (ok) return AMG_OK;
    }
  }
  AMG_TRY(gj_inverse<double>(h, h->ainv, st));
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return amg_cuda_status(e);
  return AMG_OK;
}
