// Grouped FP64 GEMM for the TEBD contractions (complex) and the eigenvector
// orthonormalisation (real).
//
// On this GPU the FP64 pipe issues about two DFMA per clock per SM, so a tile
// of 64 x 64 outputs over a reduction slab of 16 does ~256 complex MACs per
// element loaded: the kernel is bound by DFMA issue, not by memory.  One
// launch serves up to GEMM_MAXP independent problems (all triples of a
// Trotter layer), each optionally strided-batched.
#include "ptebd_internal.h"

#include <algorithm>
#include <stdexcept>

namespace ptebd {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

struct R {  // real arithmetic
  using T = double;
  static __device__ __forceinline__ T zero() { return 0.0; }
  static __device__ __forceinline__ T cj(T x) { return x; }
  static __device__ __forceinline__ T scale(T x, double s) { return x * s; }
  static __device__ __forceinline__ void mac(T& acc, T a, T b) { acc = fma(a, b, acc); }
  static __device__ __forceinline__ T mul_alpha(T x, double ar, double) { return x * ar; }
  static __device__ __forceinline__ T add(T a, T b) { return a + b; }
};

struct C {  // complex arithmetic, interleaved (re, im)
  using T = double2;
  static __device__ __forceinline__ T zero() { return make_double2(0.0, 0.0); }
  static __device__ __forceinline__ T cj(T x) { return make_double2(x.x, -x.y); }
  static __device__ __forceinline__ T scale(T x, double s) { return make_double2(x.x * s, x.y * s); }
  static __device__ __forceinline__ void mac(T& acc, T a, T b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
  }
  static __device__ __forceinline__ T mul_alpha(T x, double ar, double ai) {
    return make_double2(x.x * ar - x.y * ai, x.x * ai + x.y * ar);
  }
  static __device__ __forceinline__ T add(T a, T b) { return make_double2(a.x + b.x, a.y + b.y); }
};

template <class A_, int OPA, int OPB>
__global__ void __launch_bounds__(NT) gemm_kernel(const __grid_constant__ GemmBatch gb) {
  using T = typename A_::T;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];

  const int tile = blockIdx.x;
  int pi = 0;
  while (pi + 1 < gb.nprob && tile >= gb.tile_start[pi + 1]) ++pi;
  const GemmProb& P = gb.p[pi];
  const int local = tile - gb.tile_start[pi];
  const int tn = (P.N + BN - 1) / BN, tm = (P.M + BM - 1) / BM;
  const int per_batch = P.herm ? tm * (tm + 1) / 2 : tm * tn;
  const int bidx = local / per_batch, r = local % per_batch;
  int bm, bn;
  if (P.herm) {  // r enumerates the lower-triangular tiles row by row
    bm = (int)((sqrt(8.0 * r + 1.0) - 1.0) * 0.5);
    while (bm * (bm + 1) / 2 > r) --bm;
    while ((bm + 1) * (bm + 2) / 2 <= r) ++bm;
    bn = r - bm * (bm + 1) / 2;
  } else {
    bm = r / tn;
    bn = r % tn;
  }
  const T* __restrict__ A = static_cast<const T*>(P.A) + (long long)bidx * P.sA;
  const T* __restrict__ B = static_cast<const T*>(P.B) + (long long)bidx * P.sB;
  T* __restrict__ Cm = static_cast<T*>(P.C) + (long long)bidx * P.sC;

  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = A_::zero();

  for (int k0 = 0; k0 < P.K; k0 += BK) {
    for (int l = threadIdx.x; l < BM * BK; l += NT) {
      int i, kk;
      if (OPA == OP_C) { i = l % BM; kk = l / BM; } else { kk = l % BK; i = l / BK; }
      const int gi = bm * BM + i, gk = k0 + kk;
      T v = A_::zero();
      if (gi < P.M && gk < P.K) {
        if (OPA == OP_N) v = A[(long long)gi * P.lda + gk];
        else if (OPA == OP_C) v = A_::cj(A[(long long)gk * P.lda + gi]);
        else v = A_::cj(A[(long long)gi * P.lda + gk]);
        if (P.s_red) v = A_::scale(v, P.s_red[gk / P.red_div]);
      }
      As[kk][i] = v;
    }
    for (int l = threadIdx.x; l < BN * BK; l += NT) {
      int j, kk;
      if (OPB == OP_C) { kk = l % BK; j = l / BK; } else { j = l % BN; kk = l / BN; }
      const int gj = bn * BN + j, gk = k0 + kk;
      T v = A_::zero();
      if (gj < P.N && gk < P.K) {
        if (OPB == OP_N) v = B[(long long)gk * P.ldb + gj];
        else if (OPB == OP_C) v = A_::cj(B[(long long)gj * P.ldb + gk]);
        else v = A_::cj(B[(long long)gk * P.ldb + gj]);
        if (P.s_red_b) v = A_::scale(v, P.s_red_b[gk / P.red_div]);
      }
      Bs[kk][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) A_::mac(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }

#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gi = bm * BM + ty + 16 * i;
    if (gi >= P.M) continue;
    const double sr = P.s_row ? P.s_row[gi / P.row_div] : 1.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gj = bn * BN + tx + 16 * j;
      if (gj >= P.N) continue;
      const double sc = P.s_col ? P.s_col[gj / P.col_div] : 1.0;
      T v = A_::scale(A_::mul_alpha(acc[i][j], P.alpha_re, P.alpha_im), sr * sc);
      T* dst = Cm + (long long)gi * P.ldc + gj;
      *dst = P.accumulate ? A_::add(*dst, v) : v;
      if (P.herm && bn < bm) {  // mirror an off-diagonal tile into the upper triangle
        T* mir = Cm + (long long)gj * P.ldc + gi;
        const T cv = A_::cj(v);
        *mir = P.accumulate ? A_::add(*mir, cv) : cv;
      }
    }
  }
}

template <class A_>
void dispatch(const GemmBatch& gb, int tiles, cudaStream_t s) {
  const int key = gb.opA * 3 + gb.opB;
  switch (key) {
#define CASE(a, b) \
  case a * 3 + b: gemm_kernel<A_, a, b><<<tiles, NT, 0, s>>>(gb); break;
    CASE(0, 0) CASE(0, 1) CASE(0, 2) CASE(1, 0) CASE(1, 1) CASE(1, 2) CASE(2, 0) CASE(2, 1) CASE(2, 2)
#undef CASE
    default: throw std::runtime_error("bad gemm op");
  }
}

}  // namespace

static_assert(sizeof(GemmBatch) < 4000, "kernel parameter block too large");

GemmProb& Gemm::add(int M, int N, int K, const void* A, long long lda, const void* B, long long ldb, void* C,
                    long long ldc) {
  GemmProb p{};
  p.A = A; p.B = B; p.C = C;
  p.lda = lda; p.ldb = ldb; p.ldc = ldc;
  p.M = M; p.N = N; p.K = K; p.batch = 1;
  p.red_div = p.row_div = p.col_div = 1;
  p.alpha_re = 1.0; p.alpha_im = 0.0;
  probs_.push_back(p);
  return probs_.back();
}

int gemm_launch_single(bool complex_, int opA, int opB, const GemmProb& p, cudaStream_t s) {
  if (p.M <= 0 || p.N <= 0 || p.batch <= 0) return 0;
  GemmBatch gb{};
  gb.opA = opA;
  gb.opB = opB;
  gb.nprob = 1;
  gb.p[0] = p;
  gb.tile_start[0] = 0;
  const int tm = (p.M + BM - 1) / BM;
  gb.tile_start[1] = p.batch * (p.herm ? tm * (tm + 1) / 2 : tm * ((p.N + BN - 1) / BN));
  if (complex_) dispatch<C>(gb, gb.tile_start[1], s); else dispatch<R>(gb, gb.tile_start[1], s);
  return 1;
}

int Gemm::launch(cudaStream_t s, bool mixed, int* status) {
  if (mixed && cplx_ && opA_ == OP_N && (opB_ == OP_N || opB_ == OP_C)) {
    std::vector<TcGemmProb> tp;
    bool eligible = true;
    for (const GemmProb& p : probs_) {
      if (p.s_red || p.s_red_b || p.s_row || p.s_col || p.accumulate || p.herm || p.alpha_im != 0.0)
        eligible = false;
      TcGemmProb q{};
      q.A = static_cast<const double2*>(p.A);
      q.B = static_cast<const double2*>(p.B);
      q.C = static_cast<double2*>(p.C);
      q.lda = p.lda; q.ldb = p.ldb; q.ldc = p.ldc;
      q.sA = p.sA; q.sB = p.sB; q.sC = p.sC;
      q.alpha = p.alpha_re;
      q.M = p.M; q.N = p.N; q.K = p.K; q.batch = p.batch; q.opB = opB_;
      tp.push_back(q);
    }
    if (eligible) {
      probs_.clear();
      return tc_gemm_launch(tp, status, s);
    }
  }
  int launches = 0;
  size_t i = 0;
  while (i < probs_.size()) {
    GemmBatch gb{};
    gb.opA = opA_; gb.opB = opB_;
    int tiles = 0;
    while (i < probs_.size() && gb.nprob < GEMM_MAXP) {
      const GemmProb& p = probs_[i++];
      if (p.M <= 0 || p.N <= 0 || p.batch <= 0) continue;
      gb.p[gb.nprob] = p;
      gb.tile_start[gb.nprob] = tiles;
      const int tm = (p.M + BM - 1) / BM;
      tiles += p.batch * (p.herm ? tm * (tm + 1) / 2 : tm * ((p.N + BN - 1) / BN));
      gb.nprob++;
    }
    gb.tile_start[gb.nprob] = tiles;
    if (tiles == 0) continue;
    if (cplx_) dispatch<C>(gb, tiles, s); else dispatch<R>(gb, tiles, s);
    ++launches;
  }
  probs_.clear();
  return launches;
}

}  // namespace ptebd
