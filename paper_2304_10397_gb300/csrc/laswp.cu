// laswp.cu -- RS phase (Sec. I, Fig. 2c): apply a panel's row interchanges.
//
// The nb interchanges of a panel are sequential (row k <-> row ipiv[k]-1, k
// increasing), but their product only moves the nb rows of the panel's
// diagonal block ("top" rows) and at most nb rows below it.  A one-warp kernel
// composes them once into that permutation; the apply kernel then moves each
// touched element exactly once per column: it gathers the sources of a column
// into shared memory and scatters them to their destinations, with the top
// block written as consecutive rows (coalesced; double2 stores when aligned).
//
// perm layout (int32): [0] = q (number of displaced rows outside the top
// block), [1] = T0 (first top row, local), [2 .. 2+jb) = source row of top row
// T0+i, [2+jb .. 2+jb+q) = displaced destination rows, [2+2jb .. 2+2jb+q) =
// their source rows.  All rows are local to the matrix pointer given to apply.
#include "common.cuh"

namespace hplgb {

namespace {

constexpr int kMaxJb = 1024;

// One warp composes the jb interchanges.  The pivot rows are first read into
// shared memory in one coalesced pass (a sequential read per interchange is a
// dependent global load each, and was the kernel's whole cost); every
// interchange then finds, in parallel over the lanes, whether its row lies
// outside the top block and, if so, the slot of that row in the list of
// displaced rows (slots in order of first appearance); lane 0 finally applies
// the swaps in order, which is the only sequential part.
struct ComposeSmem {
  int32_t top[kMaxJb];
  int32_t orow[kMaxJb];
  int32_t ocont[kMaxJb];
  int32_t piv[kMaxJb];   // row of interchange t (t in application order)
  int32_t slot[kMaxJb];  // displaced-row slot of interchange t, or -1
};

// One warp: the composition into S (top: source row of each top row; orow /
// ocont: the displaced destination rows and their sources).  Returns the
// number of displaced rows, or -1 (dev_err set) for a pivot outside the rows.
__device__ int compose_warp(const int32_t* __restrict__ ipiv, int64_t k1, int64_t k2, int64_t val_shift,
                            int64_t nrows, int reverse, ComposeSmem& S, int* __restrict__ dev_err) {
  int32_t* top = S.top;
  int32_t* orow = S.orow;
  int32_t* ocont = S.ocont;
  int32_t* piv = S.piv;
  int32_t* slot = S.slot;
  const int lane = threadIdx.x & 31;
  const int jb = (int)(k2 - k1);
  const int64_t T0 = k1;  // interchange k moves row k
  int bad = 0;
  for (int t = lane; t < jb; t += 32) {
    const int64_t k = reverse ? (k2 - 1 - t) : (k1 + t);
    const int64_t p = (int64_t)ipiv[k] - 1 - val_shift;
    if (p < 0 || p >= nrows) bad = 1;
    piv[t] = (int32_t)(bad ? 0 : p);
    top[t] = (int32_t)(T0 + t);
  }
  if (__any_sync(0xffffffffu, bad)) {  // not a valid row: move nothing, report
    if (lane == 0) atomicCAS(dev_err, (int)DEV_OK, (int)DEV_BADPIV);  // a recorded timeout stays
    return -1;
  }
  __syncwarp();
  // first[t]: the first interchange s <= t naming the same row, for rows
  // outside the top block; a row is new at its first appearance
  constexpr int kPer = kMaxJb / 32;
  int isnew[kPer];
  int cnt = 0;
  const int t0 = lane * ((jb + 31) / 32);
  const int t1 = min(jb, t0 + (jb + 31) / 32);
#pragma unroll 1
  for (int t = t0; t < t1; ++t) {
    const int32_t p = piv[t];
    int fresh = 0;
    if (!(p >= T0 && p < T0 + jb)) {
      int s = 0;
      while (piv[s] != p) ++s;  // terminates at s = t at the latest
      fresh = (s == t);
      slot[t] = -(s + 2);       // provisional: -(first + 2); resolved below
    } else {
      slot[t] = -1;
    }
    isnew[t - t0] = fresh;
    cnt += fresh;
  }
  // exclusive prefix of the new-row counts over the lanes' consecutive ranges
  int incl = cnt;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += v;
  }
  const int no = __shfl_sync(0xffffffffu, incl, 31);
  int next = incl - cnt;
#pragma unroll 1
  for (int t = t0; t < t1; ++t) {
    if (isnew[t - t0]) {
      orow[next] = piv[t];
      ocont[next] = piv[t];
      slot[t] = next;  // a row's first appearance carries its slot
      ++next;
    }
  }
  __syncwarp();
  // later appearances take the slot of the first one
#pragma unroll 1
  for (int t = t0; t < t1; ++t) {
    const int v = slot[t];
    if (v <= -2) slot[t] = slot[-v - 2];
  }
  __syncwarp();
  if (lane == 0) {
#pragma unroll 1
    for (int t = 0; t < jb; ++t) {
      const int a = reverse ? (jb - 1 - t) : t;  // top slot of the row interchange t moves
      const int32_t p = piv[t];
      if (p == T0 + a) continue;
      int32_t* ps = slot[t] < 0 ? &top[p - T0] : &ocont[slot[t]];
      const int32_t tmp = top[a];
      top[a] = *ps;
      *ps = tmp;
    }
  }
  __syncwarp();
  return no;
}

// One warp composes the jb interchanges.  The pivot rows are first read into
// shared memory in one coalesced pass (a sequential read per interchange is a
// dependent global load each, and was the kernel's whole cost); every
// interchange then finds, in parallel over the lanes, whether its row lies
// outside the top block and, if so, the slot of that row in the list of
// displaced rows (slots in order of first appearance); lane 0 finally applies
// the swaps in order, which is the only sequential part.
__global__ void __launch_bounds__(32)
laswp_compose_kernel(const int32_t* __restrict__ ipiv, int64_t k1, int64_t k2, int64_t val_shift,
                     int64_t nrows, int reverse, int32_t* __restrict__ perm, int* __restrict__ dev_err) {
  __shared__ ComposeSmem S;
  const int lane = threadIdx.x;
  const int jb = (int)(k2 - k1);
  const int no = compose_warp(ipiv, k1, k2, val_shift, nrows, reverse, S, dev_err);
  if (no < 0) {
    if (lane == 0) perm[0] = -1;
    return;
  }
  if (lane == 0) { perm[0] = no; perm[1] = (int32_t)k1; }
  for (int i = lane; i < jb; i += 32) perm[2 + i] = S.top[i];
  for (int i = lane; i < no; i += 32) {
    perm[2 + jb + i] = S.orow[i];
    perm[2 + 2 * jb + i] = S.ocont[i];
  }
}

constexpr int kApplyWarps = 4;

// Columns warp, warp + nwarps, ... of A: the top rows T0 .. T0+jb-1 take rows
// top_src, rows out_dst take rows out_src; buf holds 2 jb doubles of the warp.
__device__ __forceinline__ void apply_columns(const int32_t* top_src, const int32_t* out_dst, const int32_t* out_src,
                                              int jb, int q, int64_t T0, int64_t ncols, double* __restrict__ A,
                                              int64_t lda, double* buf, int64_t warp, int64_t nwarps) {
  const int lane = threadIdx.x & 31;
  for (int64_t c = warp; c < ncols; c += nwarps) {
    double* col = A + c * lda;
    for (int i = lane; i < jb; i += 32) buf[i] = col[top_src[i]];
    for (int i = lane; i < q; i += 32) buf[jb + i] = col[out_src[i]];
    __syncwarp();
    double* topp = col + T0;
    if ((reinterpret_cast<uintptr_t>(topp) & 15) == 0 && (jb & 1) == 0) {
      double2* t2 = reinterpret_cast<double2*>(topp);
      for (int i = lane; i < (jb >> 1); i += 32) t2[i] = make_double2(buf[2 * i], buf[2 * i + 1]);
    } else {
      for (int i = lane; i < jb; i += 32) topp[i] = buf[i];
    }
    for (int i = lane; i < q; i += 32) col[out_dst[i]] = buf[jb + i];
    __syncwarp();
  }
}

// Warp per column (grid-stride).  Shared memory: the permutation plus a
// staging buffer of 2*jb doubles per warp.
__global__ void __launch_bounds__(kApplyWarps * 32)
laswp_apply_kernel(const int32_t* __restrict__ perm, int jb, int64_t ncols, double* __restrict__ A,
                   int64_t lda) {
  extern __shared__ double smem_d[];
  double* buf = smem_d + (threadIdx.x >> 5) * (2 * jb);
  int32_t* sp = reinterpret_cast<int32_t*>(smem_d + kApplyWarps * 2 * jb);
  const int q = perm[0];
  if (q < 0) return;  // the composition found an invalid pivot
  const int64_t T0 = perm[1];
  for (int i = threadIdx.x; i < jb + 2 * q; i += blockDim.x) {
    int src = i < jb ? 2 + i : (i < jb + q ? 2 + jb + (i - jb) : 2 + 2 * jb + (i - jb - q));
    sp[i] = perm[src];
  }
  __syncthreads();
  apply_columns(sp, sp + jb, sp + jb + q, jb, q, T0, ncols, A, lda, buf,
                blockIdx.x * (int64_t)kApplyWarps + (threadIdx.x >> 5), (int64_t)gridDim.x * kApplyWarps);
}

// Compose and apply in one launch, for few columns (the panel recursion):
// every CTA composes the interchanges itself (one warp, in shared memory),
// then its warps move their columns; no permutation goes through memory.
__global__ void __launch_bounds__(kApplyWarps * 32)
laswp_fused_kernel(const int32_t* __restrict__ ipiv, int64_t k1, int64_t k2, int64_t val_shift, int64_t nrows,
                   int reverse, int64_t ncols, double* __restrict__ A, int64_t lda, int* __restrict__ dev_err) {
  __shared__ ComposeSmem S;
  __shared__ int s_no;
  extern __shared__ double smem_d[];
  const int jb = (int)(k2 - k1);
  if (threadIdx.x < 32) {
    const int no = compose_warp(ipiv, k1, k2, val_shift, nrows, reverse, S, dev_err);
    if (threadIdx.x == 0) s_no = no;
  }
  __syncthreads();
  const int q = s_no;
  if (q < 0) return;
  apply_columns(S.top, S.orow, S.ocont, jb, q, k1, ncols, A, lda, smem_d + (threadIdx.x >> 5) * (2 * jb),
                blockIdx.x * (int64_t)kApplyWarps + (threadIdx.x >> 5), (int64_t)gridDim.x * kApplyWarps);
}

}  // namespace

int launch_laswp_compose(const int32_t* ipiv, int64_t k1, int64_t k2, int64_t val_shift,
                         int64_t nrows, bool reverse, int32_t* perm, int* dev_err, cudaStream_t s) {
  if (k2 - k1 > kMaxJb) return set_error(HPL_ERR_NOTSUP, "laswp: more than %d interchanges", kMaxJb);
  if (k2 <= k1) return HPL_OK;
  if (k1 < 0 || k2 > nrows) return set_error(HPL_ERR_NOTSUP, "laswp: interchange rows outside the matrix");
  laswp_compose_kernel<<<1, 32, 0, s>>>(ipiv, k1, k2, val_shift, nrows, reverse ? 1 : 0, perm, dev_err);
  count_launch();
  return check_launch("laswp_compose_kernel");
}

int launch_laswp_fused(const int32_t* ipiv, int64_t k1, int64_t k2, int64_t val_shift, int64_t nrows,
                       bool reverse, int64_t ncols, double* A, int64_t lda, int* dev_err, cudaStream_t s) {
  const int64_t jb = k2 - k1;
  if (jb > kMaxJb) return set_error(HPL_ERR_NOTSUP, "laswp: more than %d interchanges", kMaxJb);
  if (jb <= 0 || ncols <= 0) return HPL_OK;
  if (k1 < 0 || k2 > nrows) return set_error(HPL_ERR_NOTSUP, "laswp: interchange rows outside the matrix");
  const size_t smem = (size_t)kApplyWarps * 2 * jb * sizeof(double);
  HPL_TRY(set_smem_attr((const void*)laswp_fused_kernel, (int)((size_t)kApplyWarps * 2 * kMaxJb * sizeof(double))));
  const int64_t blocks = (ncols + kApplyWarps - 1) / kApplyWarps;
  laswp_fused_kernel<<<(unsigned)blocks, kApplyWarps * 32, smem, s>>>(ipiv, k1, k2, val_shift, nrows, reverse ? 1 : 0,
                                                                      ncols, A, lda, dev_err);
  count_launch();
  return check_launch("laswp_fused_kernel");
}

int launch_laswp_apply(const int32_t* perm, int64_t jb, int64_t ncols, double* A, int64_t lda,
                       cudaStream_t s) {
  if (jb <= 0 || ncols <= 0) return HPL_OK;
  size_t smem = (size_t)kApplyWarps * 2 * jb * sizeof(double) + (size_t)3 * jb * sizeof(int32_t);
  HPL_TRY(set_smem_attr((const void*)laswp_apply_kernel,
                        (int)((size_t)kApplyWarps * 2 * kMaxJb * sizeof(double) + (size_t)3 * kMaxJb * sizeof(int32_t))));
  int64_t blocks = (ncols + kApplyWarps - 1) / kApplyWarps;
  if (blocks > 152 * 32) blocks = 152 * 32;
  laswp_apply_kernel<<<(unsigned)blocks, kApplyWarps * 32, smem, s>>>(perm, (int)jb, ncols, A, lda);
  count_launch();
  return check_launch("laswp_apply_kernel");
}

}  // namespace hplgb
