// mxp_trinv.cu -- X = L11^-1 and Y = U11^-1 of a factored jb x jb diagonal
// block (packed L\U in FP32: L unit lower below the diagonal, U upper), the
// operators that turn the rest of a mixed-precision panel and its U12 block
// row into products on the tensor cores.
//
// Recursive doubling over 32-column blocks, in log2(jb / 32) levels of batched
// FP32 products instead of one serial sweep.  A node of the recursion splits
// its blocks [lo, hi) at mid = lo + ceil((hi - lo) / 2) into A = [lo, mid)
// and C = [mid, hi); with the inverses of A and C known,
//   L^-1(C, A) = -C^-1 (L(C, A) A^-1)       (A, C the blocks of L)
//   U^-1(A, C) = -(A^-1 U(A, C)) C^-1       (A, C the blocks of U)
// so the nodes of one depth, all disjoint, take two launches: the inner
// product into a jb x jb work matrix at the node's own position, then the
// outer one into X or Y.  The leaves (32 x 32 diagonal blocks) are inverted
// by substitution on [T | I], one warp per triangle; the same launch writes
// the zero triangles of X and Y, which the later products read as operands
// (the triangular operand of each product is read as a full tile).
#include <algorithm>
#include <utility>
#include <vector>

#include "common.cuh"

namespace hplgb {

namespace {

constexpr int kLB = 32;  // leaf block
constexpr int kTM = 64, kTN = 64, kTK = 16;
constexpr int kMaxNodes = 32;  // internal nodes of one depth for jb <= 2048

struct TrinvLevel {
  int nnode;
  int lo[kMaxNodes], mid[kMaxNodes], hi[kMaxNodes];  // element offsets; hi clipped to jb
};

// The tiles of one launch (both triangles), longest K first, so that the
// block scheduler pairs long tiles with short ones: node | ti << 6 | tj << 12
// | upper << 18.
constexpr int kMaxItems = 512;  // two triangles x 16 x 16 tiles at jb = 2048
struct TrinvOrder {
  uint32_t item[kMaxItems];
};

struct TrinvArgs {
  int jb;
  const float* D;  // packed L\U (ldd)
  int64_t ldd;
  float* X;  // L^-1 (ld jb)
  float* Y;  // U^-1 (ld jb)
  float* WL;  // work: L(C, A) A^-1 at (C, A) (ld jb)
  float* WU;  // work: A^-1 U(A, C) at (A, C) (ld jb)
};

// Leaf p: X(b:e, b:e) = L_pp^-1, Y(b:e, b:e) = U_pp^-1 (warps 0 and 1 of
// blockIdx.y = 0), and the zeros of column block p, X above the diagonal
// block and Y below it, spread over the kLeafSplit CTAs of the column block.
constexpr int kLeafSplit = 8;
__global__ void __launch_bounds__(256) trinv_leaf_kernel(TrinvArgs a) {
  __shared__ float T[kLB][kLB + 1];
  const int p = blockIdx.x, b = p * kLB, w = min(kLB, a.jb - b), e = b + w;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t ld = a.jb;
  const int ts = blockIdx.y * blockDim.x + t, tstride = kLeafSplit * blockDim.x;
  for (int c = 0; c < w; ++c) {
    float* xc = a.X + (int64_t)(b + c) * ld;
    float* yc = a.Y + (int64_t)(b + c) * ld;
    for (int r = ts; r < b; r += tstride) xc[r] = 0.0f;
    for (int r = e + ts; r < a.jb; r += tstride) yc[r] = 0.0f;
  }
  if (blockIdx.y != 0) return;
  for (int idx = t; idx < kLB * kLB; idx += blockDim.x) {
    const int r = idx & 31, c = idx >> 5;
    T[r][c] = (r < w && c < w) ? a.D[b + r + (int64_t)(b + c) * a.ldd] : (r == c ? 1.0f : 0.0f);
  }
  __syncthreads();
  if (warp == 0) {  // row `lane` of U^-1 by back substitution on [U | I]
    float v[kLB];
#pragma unroll
    for (int c = 0; c < kLB; ++c) v[c] = lane == c ? 1.0f : 0.0f;
    const float rd = 1.0f / T[lane][lane];
#pragma unroll 1
    for (int j = kLB - 1; j >= 0; --j) {
      const float rj = __shfl_sync(0xffffffffu, rd, j);
      const float uij = lane < j ? T[lane][j] : 0.0f;
#pragma unroll
      for (int c = 0; c < kLB; ++c) {
        const float sj = __shfl_sync(0xffffffffu, v[c], j) * rj;  // U^-1(j, c)
        v[c] = lane == j ? sj : fmaf(-uij, sj, v[c]);
      }
    }
    if (lane < w)
#pragma unroll
      for (int c = 0; c < kLB; ++c)
        if (c < w) a.Y[b + lane + (int64_t)(b + c) * ld] = v[c];
  } else if (warp == 1) {  // row `lane` of L^-1 by forward elimination on [L | I]
    float v[kLB];
#pragma unroll
    for (int c = 0; c < kLB; ++c) v[c] = lane == c ? 1.0f : 0.0f;
#pragma unroll 1
    for (int j = 0; j < kLB; ++j) {
      const float lij = lane > j ? T[lane][j] : 0.0f;
#pragma unroll
      for (int c = 0; c < kLB; ++c) v[c] = fmaf(-lij, __shfl_sync(0xffffffffu, v[c], j), v[c]);
    }
    if (lane < w)
#pragma unroll
      for (int c = 0; c < kLB; ++c)
        if (c < w) a.X[b + lane + (int64_t)(b + c) * ld] = v[c];
  }
}

// One product of one depth for every node, blockIdx.y = 0 for L, 1 for U:
//   outer = 0: WL(C, A) = L(C, A) X(A, A)      WU(A, C) = Y(A, A) U(A, C)
//   outer = 1: X(C, A) = -X(C, C) WL(C, A)     Y(A, C) = -WU(A, C) Y(C, C)
// 64 x 64 tiles, 4 x 4 outputs per thread, K in slices of 16 copied into
// shared memory by cp.async, kTS slices in flight (the operands come from L2,
// and one slice of arithmetic is shorter than its latency).  The triangular
// operand limits K per tile to where it can be nonzero.
constexpr int kTS = 4;

__host__ __device__ inline void k_range(bool upper, int outer, int i0, int j0, int K, int* klo, int* khi) {
  *klo = 0;
  *khi = K;
  if (!upper && outer == 0) *klo = j0;
  if (!upper && outer == 1) *khi = i0 + kTM < K ? i0 + kTM : K;
  if (upper && outer == 0) *klo = i0;
  if (upper && outer == 1) *khi = j0 + kTN < K ? j0 + kTN : K;
}

__device__ __forceinline__ void cp_async4_zfill(float* dst, const float* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src),
               "r"(valid ? 4 : 0)
               : "memory");
}

__global__ void __launch_bounds__(256) trinv_prod_kernel(TrinvArgs a, TrinvLevel lv, const __grid_constant__ TrinvOrder ord,
                                                         int outer) {
  __shared__ __align__(16) float Ps[kTS][kTK][kTM];
  __shared__ __align__(16) float Qs[kTS][kTK][kTN + 4];  // padded: the copies run down k
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const uint32_t it = ord.item[blockIdx.x];
  const int nd = (int)(it & 63), ti = (int)((it >> 6) & 63), tj = (int)((it >> 12) & 63);
  const bool upper = ((it >> 18) & 1) != 0;
  const int a0 = lv.lo[nd], a1 = lv.mid[nd], c1 = lv.hi[nd];
  const int sa = a1 - a0, scn = c1 - a1;
  const int64_t ld = a.jb;
  const float *P, *Q;
  int64_t ldp, ldq;
  float* O;
  int M, N, K;
  if (!upper) {
    M = scn, N = sa;
    if (outer == 0) {
      P = a.D + a1 + (int64_t)a0 * a.ldd, ldp = a.ldd;
      Q = a.X + a0 + (int64_t)a0 * ld, ldq = ld;
      O = a.WL + a1 + (int64_t)a0 * ld, K = sa;
    } else {
      P = a.X + a1 + (int64_t)a1 * ld, ldp = ld;
      Q = a.WL + a1 + (int64_t)a0 * ld, ldq = ld;
      O = a.X + a1 + (int64_t)a0 * ld, K = scn;
    }
  } else {
    M = sa, N = scn;
    if (outer == 0) {
      P = a.Y + a0 + (int64_t)a0 * ld, ldp = ld;
      Q = a.D + a0 + (int64_t)a1 * a.ldd, ldq = a.ldd;
      O = a.WU + a0 + (int64_t)a1 * ld, K = sa;
    } else {
      P = a.WU + a0 + (int64_t)a1 * ld, ldp = ld;
      Q = a.Y + a1 + (int64_t)a1 * ld, ldq = ld;
      O = a.Y + a0 + (int64_t)a1 * ld, K = scn;
    }
  }
  const int i0 = ti * kTM, j0 = tj * kTN;
  // K range where the triangular operand of this tile can be nonzero:
  //   L inner: X(A, A) lower, Q(k, j) = 0 for k < j      -> k >= j0
  //   L outer: X(C, C) lower, P(i, k) = 0 for k > i      -> k < i0 + 64
  //   U inner: Y(A, A) upper, P(i, k) = 0 for k < i      -> k >= i0
  //   U outer: Y(C, C) upper, Q(k, j) = 0 for k > j      -> k < j0 + 64
  int klo, khi;
  k_range(upper, outer, i0, j0, K, &klo, &khi);

  float acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.0f;
  // slice copies: P element (i, k) with i = t % 64, k = t / 64 + 4 r; Q element
  // (k, j) with k = t % 16, j = t / 16 + 16 r; entries outside the operands
  // (or past khi) are zero-filled
  const int nsl = klo < khi ? (khi - klo + kTK - 1) / kTK : 0;
  // P in 16-byte pieces (4 rows of one column) where the column is aligned
  const bool vecP = ((ldp & 3) == 0) && ((reinterpret_cast<uintptr_t>(P + i0) & 15) == 0);
  auto issue = [&](int sl) {
    if (sl < nsl) {
      const int k0 = klo + sl * kTK, st = sl % kTS;
      {
        const int i4 = (t & 15) * 4, k = k0 + (t >> 4), i = i0 + i4;
        float* dst = &Ps[st][t >> 4][i4];
        if (vecP && i + 3 < M && k < khi) {
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                       "l"(P + i + (int64_t)k * ldp)
                       : "memory");
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const bool vp = i + q < M && k < khi;
            cp_async4_zfill(dst + q, vp ? P + i + q + (int64_t)k * ldp : P, vp);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int kq = k0 + (t & 15), j = j0 + (t >> 4) + 16 * r;
        const bool vq = j < N && kq < khi;
        cp_async4_zfill(&Qs[st][t & 15][(t >> 4) + 16 * r], vq ? Q + kq + (int64_t)j * ldq : Q, vq);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");  // empty groups keep the count
  };
#pragma unroll
  for (int sl = 0; sl < kTS - 1; ++sl) issue(sl);
  for (int sl = 0; sl < nsl; ++sl) {
    asm volatile("cp.async.wait_group %0;" ::"n"(kTS - 2) : "memory");
    __syncthreads();  // slice sl is in; every thread is done with slice sl - 1
    issue(sl + kTS - 1);
    const int st = sl % kTS;
#pragma unroll
    for (int k = 0; k < kTK; ++k) {
      const float4 pv = *reinterpret_cast<const float4*>(&Ps[st][k][ty * 4]);
      const float4 qv = *reinterpret_cast<const float4*>(&Qs[st][k][tx * 4]);
      const float pa[4] = {pv.x, pv.y, pv.z, pv.w}, qa[4] = {qv.x, qv.y, qv.z, qv.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(pa[u], qa[v], acc[u][v]);
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  const float sg = outer ? -1.0f : 1.0f;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int j = j0 + tx * 4 + v;
    if (j >= N) continue;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + ty * 4 + u;
      if (i < M) O[i + (int64_t)j * ld] = sg * acc[u][v];
    }
  }
}

void split_nodes(int lo, int hi, int depth, std::vector<std::vector<int>>& by_depth) {
  if (hi - lo < 2) return;
  const int mid = lo + (hi - lo + 1) / 2;
  if ((int)by_depth.size() <= depth) by_depth.resize(depth + 1);
  by_depth[depth].push_back(lo);
  by_depth[depth].push_back(mid);
  by_depth[depth].push_back(hi);
  split_nodes(lo, mid, depth + 1, by_depth);
  split_nodes(mid, hi, depth + 1, by_depth);
}

}  // namespace

int trinv_work_floats(int64_t jb) { return (int)(2 * jb * jb); }

// X = L^-1 and Y = U^-1 (ld jb) of the packed factors D (jb x jb, ldd),
// jb <= 2048; wk holds trinv_work_floats(jb) floats.  A zero on U's diagonal
// gives infinities or NaNs in Y (the factorization reports it through info).
int launch_mxp_trinv(int64_t jb, const float* D, int64_t ldd, float* X, float* Y, float* wk, cudaStream_t s) {
  if (jb <= 0) return HPL_OK;
  if (jb > 2048) return set_error(HPL_ERR_NOTSUP, "triangular inverse larger than 2048");
  TrinvArgs a;
  a.jb = (int)jb;
  a.D = D;
  a.ldd = ldd;
  a.X = X;
  a.Y = Y;
  a.WL = wk;
  a.WU = wk + jb * jb;
  const int nblk = (int)((jb + kLB - 1) / kLB);
  trinv_leaf_kernel<<<dim3((unsigned)nblk, kLeafSplit), 256, 0, s>>>(a);
  count_launch();
  HPL_TRY(check_launch("trinv_leaf_kernel"));
  std::vector<std::vector<int>> by_depth;
  split_nodes(0, nblk, 0, by_depth);
  for (int d = (int)by_depth.size() - 1; d >= 0; --d) {
    const std::vector<int>& nodes = by_depth[d];
    TrinvLevel lv;
    lv.nnode = (int)nodes.size() / 3;
    if (lv.nnode > kMaxNodes) return set_error(HPL_ERR_NOTSUP, "triangular inverse: %d nodes at one depth", lv.nnode);
    for (int i = 0; i < lv.nnode; ++i) {
      lv.lo[i] = nodes[3 * i] * kLB;
      lv.mid[i] = nodes[3 * i + 1] * kLB;
      lv.hi[i] = (int)(nodes[3 * i + 2] * kLB < jb ? nodes[3 * i + 2] * kLB : jb);
    }
    for (int outer = 0; outer < 2; ++outer) {
      // every tile of both triangles with its K length, longest first
      std::vector<std::pair<int, uint32_t>> items;
      for (int up = 0; up < 2; ++up)
        for (int i = 0; i < lv.nnode; ++i) {
          const int sa = lv.mid[i] - lv.lo[i], scn = lv.hi[i] - lv.mid[i];
          const int M = up ? sa : scn, N = up ? scn : sa, K = outer == 0 ? sa : scn;
          for (int tj = 0; tj * kTN < N; ++tj)
            for (int ti = 0; ti * kTM < M; ++ti) {
              int klo, khi;
              k_range(up != 0, outer, ti * kTM, tj * kTN, K, &klo, &khi);
              items.push_back({-(khi - klo), (uint32_t)i | (uint32_t)ti << 6 | (uint32_t)tj << 12 | (uint32_t)up << 18});
            }
        }
      if ((int)items.size() > kMaxItems) return set_error(HPL_ERR_NOTSUP, "triangular inverse: %d tiles", (int)items.size());
      std::stable_sort(items.begin(), items.end(),
                       [](const std::pair<int, uint32_t>& x, const std::pair<int, uint32_t>& y) { return x.first < y.first; });
      TrinvOrder ord;
      for (size_t q = 0; q < items.size(); ++q) ord.item[q] = items[q].second;
      trinv_prod_kernel<<<(unsigned)items.size(), 256, 0, s>>>(a, lv, ord, outer);
      count_launch();
      HPL_TRY(check_launch("trinv_prod_kernel"));
    }
  }
  return HPL_OK;
}

}  // namespace hplgb
