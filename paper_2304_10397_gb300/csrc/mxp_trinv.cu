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
  int tile0[kMaxNodes + 1];                          // prefix sums of the tiles of each node
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

// Leaf p: X(b:e, b:e) = L_pp^-1, Y(b:e, b:e) = U_pp^-1 (warps 0 and 1), and
// the zeros of column block p: X above the diagonal block, Y below it.
__global__ void __launch_bounds__(256) trinv_leaf_kernel(TrinvArgs a) {
  __shared__ float T[kLB][kLB + 1];
  const int p = blockIdx.x, b = p * kLB, w = min(kLB, a.jb - b), e = b + w;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int64_t ld = a.jb;
  for (int idx = t; idx < kLB * kLB; idx += blockDim.x) {
    const int r = idx & 31, c = idx >> 5;
    T[r][c] = (r < w && c < w) ? a.D[b + r + (int64_t)(b + c) * a.ldd] : (r == c ? 1.0f : 0.0f);
  }
  for (int c = 0; c < w; ++c) {
    float* xc = a.X + (int64_t)(b + c) * ld;
    float* yc = a.Y + (int64_t)(b + c) * ld;
    for (int r = t; r < b; r += blockDim.x) xc[r] = 0.0f;
    for (int r = e + t; r < a.jb; r += blockDim.x) yc[r] = 0.0f;
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
// 64 x 64 tiles, 4 x 4 outputs per thread, K in steps of 16 staged through
// shared memory (double buffered).  The triangular operand limits K per tile
// to where it can be nonzero.
__global__ void __launch_bounds__(256) trinv_prod_kernel(TrinvArgs a, TrinvLevel lv, int outer) {
  __shared__ __align__(16) float Ps[2][kTK][kTM];
  __shared__ __align__(16) float Qs[2][kTK][kTN + 4];  // padded: the staging stores run down k
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const bool upper = blockIdx.y == 1;
  int tile = blockIdx.x, nd = 0;
  while (nd + 1 < lv.nnode && tile >= lv.tile0[nd + 1]) ++nd;
  tile -= lv.tile0[nd];
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
  const int tm = (M + kTM - 1) / kTM;
  const int i0 = (tile % tm) * kTM, j0 = (tile / tm) * kTN;
  // K range where the triangular operand of this tile can be nonzero:
  //   L inner: X(A, A) lower, Q(k, j) = 0 for k < j      -> k >= j0
  //   L outer: X(C, C) lower, P(i, k) = 0 for k > i      -> k < i0 + 64
  //   U inner: Y(A, A) upper, P(i, k) = 0 for k < i      -> k >= i0
  //   U outer: Y(C, C) upper, Q(k, j) = 0 for k > j      -> k < j0 + 64
  int klo = 0, khi = K;
  if (!upper && outer == 0) klo = j0;
  if (!upper && outer == 1) khi = min(K, i0 + kTM);
  if (upper && outer == 0) klo = i0;
  if (upper && outer == 1) khi = min(K, j0 + kTN);

  float acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.0f;
  // global -> register staging: P element (i, k) with i = t % 64, k = t / 64 + 4 r;
  // Q element (k, j) with k = t % 16, j = t / 16 + 16 r
  float pr[4], qr[4];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = i0 + (t & 63), k = k0 + (t >> 6) + 4 * r;
      pr[r] = (i < M && k < khi) ? P[i + (int64_t)k * ldp] : 0.0f;
      const int kq = k0 + (t & 15), j = j0 + (t >> 4) + 16 * r;
      qr[r] = (j < N && kq < khi) ? Q[kq + (int64_t)j * ldq] : 0.0f;
    }
  };
  auto stage = [&](int buf) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      Ps[buf][(t >> 6) + 4 * r][t & 63] = pr[r];
      Qs[buf][t & 15][(t >> 4) + 16 * r] = qr[r];
    }
  };
  int buf = 0;
  if (klo < khi) {
    fetch(klo);
    stage(0);
    __syncthreads();
    for (int k0 = klo; k0 < khi; k0 += kTK) {
      const bool more = k0 + kTK < khi;
      if (more) fetch(k0 + kTK);
#pragma unroll
      for (int k = 0; k < kTK; ++k) {
        const float4 pv = *reinterpret_cast<const float4*>(&Ps[buf][k][ty * 4]);
        const float4 qv = *reinterpret_cast<const float4*>(&Qs[buf][k][tx * 4]);
        const float pa[4] = {pv.x, pv.y, pv.z, pv.w}, qa[4] = {qv.x, qv.y, qv.z, qv.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(pa[u], qa[v], acc[u][v]);
      }
      if (more) {
        stage(buf ^ 1);
        __syncthreads();
        buf ^= 1;
      }
    }
  }
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
  trinv_leaf_kernel<<<nblk, 256, 0, s>>>(a);
  count_launch();
  HPL_TRY(check_launch("trinv_leaf_kernel"));
  std::vector<std::vector<int>> by_depth;
  split_nodes(0, nblk, 0, by_depth);
  for (int d = (int)by_depth.size() - 1; d >= 0; --d) {
    const std::vector<int>& nodes = by_depth[d];
    TrinvLevel lv;
    lv.nnode = (int)nodes.size() / 3;
    if (lv.nnode > kMaxNodes) return set_error(HPL_ERR_NOTSUP, "triangular inverse: %d nodes at one depth", lv.nnode);
    lv.tile0[0] = 0;
    for (int i = 0; i < lv.nnode; ++i) {
      lv.lo[i] = nodes[3 * i] * kLB;
      lv.mid[i] = nodes[3 * i + 1] * kLB;
      lv.hi[i] = (int)(nodes[3 * i + 2] * kLB < jb ? nodes[3 * i + 2] * kLB : jb);
      const int sa = lv.mid[i] - lv.lo[i], scn = lv.hi[i] - lv.mid[i];
      lv.tile0[i + 1] = lv.tile0[i] + ((scn + kTM - 1) / kTM) * ((sa + kTN - 1) / kTN);
    }
    for (int outer = 0; outer < 2; ++outer) {
      trinv_prod_kernel<<<dim3((unsigned)lv.tile0[lv.nnode], 2), 256, 0, s>>>(a, lv, outer);
      count_launch();
      HPL_TRY(check_launch("trinv_prod_kernel"));
    }
  }
  return HPL_OK;
}

}  // namespace hplgb
