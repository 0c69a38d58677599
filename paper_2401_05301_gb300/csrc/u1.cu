// Particle-number (U(1)) blocked form of the three-site local update.
//
// The paper runs its TEBD with U(1)-symmetric tensors (Sec. II B): every gate
// conserves the boson number N, so each Schmidt vector of bond k can carry a
// definite charge q_k(a), the number of bosons on the sites left of the bond,
// and B_k[a, s, b] vanishes unless q_{k+1}(b) = q_k(a) + s.  This file takes
// every product and both truncated SVDs of the update of Sec. II B block by
// block over those charges; the site tensors stay dense in HBM (zero outside
// their blocks), so measurement and state I/O are those of the dense form.
//
// Layout choices (a gauge: the state is unchanged):
//   * every bond's Schmidt index is kept sorted by charge, so each charge is one
//     contiguous run [st(v), st(v) + n(v)) and every block of a site tensor is a
//     plain strided matrix;
//   * theta~ and C = G theta~ are held compactly, grouped by the occupation
//     Delta = s1 + s2 + s3 = q_{i+3}(b) - q_i(a) that the gate conserves: for
//     each Delta a matrix with one row per sigma = (s1, s2, s3) of that total
//     and one column per pair (a, b) with q(b) - q(a) = Delta, so the gate is one
//     plain product per Delta;
//   * the cut of each SVD is block diagonal in its charge c; the rows and
//     columns of a block are packed into a dense matrix by affine block copies.
// Each block then goes through the engines of the dense form: Gram product,
// Householder reduction, multisection, inverse iteration, projection.  Rule T
// is applied once to the merged spectrum of all blocks of a cut (ties: block
// order, then index), and the kept vectors are ordered by charge.
#include "ptebd_ctx.h"

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <complex>
#include <cstring>
#include <functional>
#include <numeric>
#include <stdexcept>
#include <vector>

namespace ptebd {

struct U1Arena {
  char* base = nullptr;
  size_t cap = 0;
};

struct U1Slot {
  U1Arena a1, a2;  // a1: products up to the first cut's rebuild; a2: the second cut
};

struct U1Work {
  std::vector<U1Slot> slots;
  // digit workspaces of the exact-digit engine, one per problem of a launch: OZ_MAXP for
  // the block products (sized for the largest), EIG_MAXP for the eigen-solver's products
  std::vector<void*> ring, ering;
  size_t ring_bytes = 0, ering_bytes = 0;
  char* h_stage[2] = {nullptr, nullptr};  // pinned staging of descriptors, by chunk parity
  char* d_stage[2] = {nullptr, nullptr};
  size_t stage_cap[2] = {0, 0};
  size_t stage_used = 0;
  int parity = 0;
  cudaEvent_t ev[2] = {nullptr, nullptr};  // last use of each staging buffer
  std::vector<std::pair<char*, char*>> retired[2];  // outgrown staging buffers, freed once idle
  double* h_back = nullptr;                // pinned read-back buffer
  size_t h_back_n = 0;
  U1Arena meas;                            // blocks of the correlator products
  int* d_counts = nullptr;                 // eigenvalues needed per block of a batch of cuts
  size_t d_counts_n = 0;
};

namespace {

constexpr int RING = OZ_MAXP;    // problems of one exact-digit launch
constexpr int ERING = EIG_MAXP;  // matrices of one eigen-solver batch
constexpr int MV_TILE = 4096;   // elements per block of the move kernel
constexpr int TR_THREADS = 1024;

// ---- kernels ----------------------------------------------------------------------

// One affine block copy between a strided view and a packed block.
struct Move {
  void* sv;  // strided view: element (i, j) at sv[i * rs + j * cs]
  void* pk;  // packed block: element (i, j) at pk[i * ldp + j]
  long long rs, cs, ldp;
  int rows, cols;
  int dir;   // 0: gather (view -> packed), 1: scatter (packed -> view)
  int real;  // elements are doubles instead of complex doubles
};

__global__ void k_move(const Move* __restrict__ mv, const long long* __restrict__ tile_start, int nmv) {
  // the move this block serves: last m with tile_start[m] <= blockIdx.x
  int lo = 0, hi = nmv - 1;
  const long long t = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tile_start[mid] <= t) lo = mid; else hi = mid - 1;
  }
  const Move m = mv[lo];
  const long long total = (long long)m.rows * m.cols;
  const long long e0 = (t - tile_start[lo]) * MV_TILE;
  const long long e1 = min(total, e0 + MV_TILE);
  for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const long long i = e / m.cols, j = e - i * m.cols;
    const long long so = i * m.rs + j * m.cs, po = i * m.ldp + j;
    if (m.real) {
      double* sv = static_cast<double*>(m.sv);
      double* pk = static_cast<double*>(m.pk);
      if (m.dir == 0) pk[po] = sv[so]; else sv[so] = pk[po];
    } else {
      double2* sv = static_cast<double2*>(m.sv);
      double2* pk = static_cast<double2*>(m.pk);
      if (m.dir == 0) pk[po] = sv[so]; else sv[so] = pk[po];
    }
  }
}

// Candidates of one cut: the rows of Y_c = u_k^+ theta'_c of every charge block.
struct TruncBlk {
  const double2* Y;
  int K, n;
};

struct TruncCut {
  const TruncBlk* blk;  // blocks in ascending charge order
  int nb, ncand;        // blocks, sum of K
  double total;         // ||theta'||^2: sum of the blocks' Gram traces
  int chi_max;
  double w_cut, eps_rel;
  double* lam_out;  // [chi'] kept s / ||s_kept||, in (block, row) order
  double* s_out;    // [chi'] kept s
  int* row_out;     // [chi'] row of the kept value in its block's Y
  int* counts;      // [nb] kept values per block
  int* chi_out;
  double* norm_out;
  double* w_out;
  int* status;
};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return __shfl_sync(0xffffffffu, v, 0);
}

// Bitonic sort of (s, key) over P entries (P a power of two): descending s with
// ascending key on ties (desc_s), or ascending key (otherwise).
__device__ void bitonic(double* s, int* key, int P, bool desc_s) {
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int jx = i ^ stride;
        if (jx > i) {
          const bool up = ((i & size) == 0);
          const double si = s[i], sj = s[jx];
          const int ki = key[i], kj = key[jx];
          const bool i_first = desc_s ? ((si > sj) || (si == sj && ki < kj)) : (ki < kj);
          if (up != i_first) { s[i] = sj; s[jx] = si; key[i] = kj; key[jx] = ki; }
        }
      }
      __syncthreads();
    }
  }
}

// Rule T (the tolerances of Sec. II B) on the merged spectrum of one cut:
// p_k = s_k^2 / total, chi_w = smallest k with sum_{i>k} p_i <= w_cut,
// chi_eps = #{p_k > eps_rel}, chi' = max(1, min(chi_max, chi_w, chi_eps, K)); the
// tail beyond the computed values is total - sum s^2.  The kept values are then
// re-ordered by (block, row) so that the new bond is sorted by charge.
__global__ void __launch_bounds__(TR_THREADS) k_trunc_u1(const TruncCut* __restrict__ cuts) {
  const TruncCut& A = cuts[blockIdx.x];
  extern __shared__ unsigned char smem_raw[];
  int P = 1;
  while (P < A.ncand) P <<= 1;
  double* s = reinterpret_cast<double*>(smem_raw);
  int* key = reinterpret_cast<int*>(s + P);
  __shared__ int off[1025];
  __shared__ int cnt_sh[1024];
  __shared__ int chi_sh;
  __shared__ double norm_sh;
  if (threadIdx.x == 0) {
    int o = 0;
    for (int b = 0; b < A.nb; ++b) { off[b] = o; o += A.blk[b].K; }
    off[A.nb] = o;
  }
  for (int b = threadIdx.x; b < A.nb; b += blockDim.x) cnt_sh[b] = 0;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int g = warp; g < A.ncand; g += nw) {
    int b = 0;
    while (off[b + 1] <= g) ++b;
    const TruncBlk& T = A.blk[b];
    const double2* y = T.Y + (size_t)(g - off[b]) * T.n;
    double acc = 0.0;
    for (int c = lane; c < T.n; c += 32) acc = fma(y[c].x, y[c].x, fma(y[c].y, y[c].y, acc));
    acc = warp_sum_d(acc);
    if (lane == 0) { s[g] = sqrt(acc); key[g] = g; }
  }
  for (int g = A.ncand + threadIdx.x; g < P; g += blockDim.x) { s[g] = -1.0; key[g] = 0x7fffffff; }
  __syncthreads();
  bitonic(s, key, P, true);
  if (threadIdx.x == 0) {
    const double total = A.total;
    const int K = A.ncand;
    bool bad = !(total > 0.0) || !isfinite(total);
    double sumK = 0.0;
    for (int i = 0; i < K; ++i) {
      if (!isfinite(s[i])) bad = true;
      sumK += s[i] * s[i];
    }
    int chi = 1;
    double w = 0.0, kept = (K > 0) ? s[0] * s[0] : 0.0;
    if (!bad) {
      const double tailK = fmax(0.0, total - sumK);
      int chi_eps = 0;
      for (int i = 0; i < K; ++i) chi_eps += (s[i] * s[i] / total > A.eps_rel);
      chi_eps = max(chi_eps, 1);
      const double thr = A.w_cut * total;
      int chi_w = K;
      double tail = tailK;
      for (int k = K; k >= 1; --k) {
        if (tail <= thr) chi_w = k; else break;
        tail += s[k - 1] * s[k - 1];
      }
      chi = max(1, min(min(A.chi_max, chi_w), min(chi_eps, K)));
      double tc = tailK;
      for (int i = K - 1; i >= chi; --i) tc += s[i] * s[i];
      w = tc / total;
      kept = 0.0;
      for (int i = 0; i < chi; ++i) kept += s[i] * s[i];
    } else {
      atomicExch(A.status, TEBD_ERR_NONFINITE);
    }
    chi_sh = chi;
    norm_sh = sqrt(kept);
    *A.chi_out = chi;
    *A.norm_out = norm_sh;
    *A.w_out = w;
  }
  __syncthreads();
  const int chi = chi_sh;
  // the kept entries by (block, row): sort the first chi entries by key
  int P2 = 1;
  while (P2 < chi) P2 <<= 1;
  for (int g = chi + threadIdx.x; g < P2; g += blockDim.x) { s[g] = -1.0; key[g] = 0x7fffffff; }
  __syncthreads();
  bitonic(s, key, P2, false);
  const double inv = (norm_sh > 0.0) ? 1.0 / norm_sh : 0.0;
  for (int k = threadIdx.x; k < chi; k += blockDim.x) {
    const int g = key[k];
    int b = 0;
    while (off[b + 1] <= g) ++b;
    A.lam_out[k] = s[k] * inv;
    A.s_out[k] = s[k];
    A.row_out[k] = g - off[b];
    atomicAdd(&cnt_sh[b], 1);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < A.nb; b += blockDim.x) A.counts[b] = cnt_sh[b];
}

// V_c[i, :] = Y_c[row[kst + i], :] / s[kst + i] and W_c = 1.5 V_c (the first term
// of the Newton-Schulz step W = 1.5 V - 0.5 (V V^+) V).
struct KeptGather {
  const double2* Y;
  double2* V;
  double2* W;
  const int* row;
  const double* s;
  int n, kst, cnt;
};

__global__ void k_kept_gather(const KeptGather* __restrict__ kg) {
  const KeptGather G = kg[blockIdx.y];
  const int i = blockIdx.x;
  if (i >= G.cnt) return;
  const double2* src = G.Y + (size_t)G.row[G.kst + i] * G.n;
  const double sv = G.s[G.kst + i];
  const double inv = (sv > 0.0) ? 1.0 / sv : 0.0;
  for (int j = threadIdx.x; j < G.n; j += blockDim.x) {
    const double2 v = src[j];
    const double2 x = make_double2(v.x * inv, v.y * inv);
    G.V[(size_t)i * G.n + j] = x;
    G.W[(size_t)i * G.n + j] = make_double2(1.5 * x.x, 1.5 * x.y);
  }
}

// Blocks decomposed from the right Gram matrix: U holds the right singular vectors z_k
// (K rows of length n).  The rows the truncation expects are Y_k = s_k z_k^+, with
// s_k = ||lam P z_k|| (second-order accurate in the eigenvector error, like the row norms
// of the left projection) from T = (lam P) [z_0 .. z_{K-1}] (b x K).
struct RightRows {
  const double2* U;
  double2* Y;
  const double2* T;
  int K, n, b;
};

// Y = conj(U): the rows z_k^+ (also the second operand of T = (lam P) Y^+)
__global__ void k_right_conj(const RightRows* __restrict__ rr) {
  const RightRows R = rr[blockIdx.y];
  const int k = blockIdx.x;
  if (k >= R.K) return;
  for (int j = threadIdx.x; j < R.n; j += blockDim.x) {
    const double2 u = R.U[(size_t)k * R.n + j];
    R.Y[(size_t)k * R.n + j] = make_double2(u.x, -u.y);
  }
}

// Y_k *= ||T[:, k]||
__global__ void k_right_scale(const RightRows* __restrict__ rr) {
  __shared__ double sh[32];
  __shared__ double s_sh;
  const RightRows R = rr[blockIdx.y];
  const int k = blockIdx.x;
  if (k >= R.K) return;
  double acc = 0.0;
  for (int r = threadIdx.x; r < R.b; r += blockDim.x) {
    const double2 t = R.T[(size_t)r * R.K + k];
    acc = fma(t.x, t.x, fma(t.y, t.y, acc));
  }
  acc = warp_sum_d(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    s_sh = sqrt(t);
  }
  __syncthreads();
  const double sk = s_sh;
  for (int j = threadIdx.x; j < R.n; j += blockDim.x) {
    double2& y = R.Y[(size_t)k * R.n + j];
    y = make_double2(sk * y.x, sk * y.y);
  }
}

// f[i] = lam[i]^2 w[i] (the reduction factors of the correlator's left product)
__global__ void k_lam2w(const double* __restrict__ lam, const double* __restrict__ w, double* __restrict__ f, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) f[i] = lam[i] * lam[i] * w[i];
}

// The gate on the compact theta~: C_Delta = G_Delta theta~_Delta for every conserved
// total Delta, G_Delta an nd x nd block (nd <= 48 for d <= 8) and theta~_Delta nd x N
// (row stride N).  A thread takes one column: the nd entries in registers, G in shared
// memory (read by all lanes at once), the nd outputs accumulated in sigma order.  The
// reduction is too short for the tensor cores' accumulation (a single k-step), so the
// product stays on the FP64 pipe, with no padding of the small dimension.
struct GateBlk {
  const double2* G;
  const double2* X;
  double2* C;
  long long N;
  int nd;
  int blk0;  // first block of this problem in the launch
};

template <int NDM>
__global__ void __launch_bounds__(128) k_gate_blocks(const GateBlk* __restrict__ gb, int nprob) {
  __shared__ double2 Gs[NDM * NDM];
  int lo = 0, hi = nprob - 1;  // the problem whose blocks hold blockIdx.x
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (gb[mid].blk0 <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const GateBlk P = gb[lo];
  const int nd = P.nd;
  for (int e = threadIdx.x; e < nd * nd; e += blockDim.x) Gs[e] = P.G[e];
  __syncthreads();
  const long long j = (long long)(blockIdx.x - P.blk0) * blockDim.x + threadIdx.x;
  if (j >= P.N) return;
  double2 x[NDM];
#pragma unroll
  for (int q = 0; q < NDM; ++q) x[q] = (q < nd) ? P.X[(long long)q * P.N + j] : make_double2(0.0, 0.0);
  for (int r = 0; r < nd; ++r) {
    double re = 0.0, im = 0.0;
    const double2* g = Gs + r * nd;
#pragma unroll
    for (int q = 0; q < NDM; ++q) {
      if (q < nd) {
        const double2 a = g[q];
        re = fma(a.x, x[q].x, fma(-a.y, x[q].y, re));
        im = fma(a.x, x[q].y, fma(a.y, x[q].x, im));
      }
    }
    P.C[(long long)r * P.N + j] = make_double2(re, im);
  }
}

// One bond's correlator from its charge blocks: out[bond] = sum over its blocks v of
// sum_{i, j} X_v[i][j] Y_v[j][i] (X_v: nu x nv, Y_v: nv x nu), in a fixed order.
struct TraceBlk {
  const double2* X;
  const double2* Y;
  int nu, nv;
};
struct TraceBond {
  int b0, b1;  // blocks [b0, b1) of the list
  double2* out;
};

__global__ void k_trace_bonds(const TraceBond* __restrict__ bonds, const TraceBlk* __restrict__ blk) {
  const TraceBond B = bonds[blockIdx.x];
  __shared__ double re_sh[32], im_sh[32];
  double re = 0.0, im = 0.0;
  for (int q = B.b0; q < B.b1; ++q) {
    const TraceBlk T = blk[q];
    const int n = T.nu * T.nv;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const int i = e / T.nv, j = e - i * T.nv;
      const double2 x = T.X[(size_t)i * T.nv + j], y = T.Y[(size_t)j * T.nu + i];
      re = fma(x.x, y.x, fma(-x.y, y.y, re));
      im = fma(x.x, y.y, fma(x.y, y.x, im));
    }
  }
  re = warp_sum_d(re);
  im = warp_sum_d(im);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { re_sh[w] = re; im_sh[w] = im; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0, m = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { r += re_sh[k]; m += im_sh[k]; }
    *B.out = make_double2(r, m);
  }
}

// ---- host: charges ------------------------------------------------------------------

struct Runs {  // charge v occupies [st[v - q0], st[v - q0] + n[v - q0]) of the bond index
  int q0 = 0;
  std::vector<int> st, n;
  int count(int v) const {
    const int k = v - q0;
    return (k >= 0 && k < (int)n.size()) ? n[k] : 0;
  }
  int start(int v) const { return st[v - q0]; }
  int lo() const { return q0; }
  int hi() const { return q0 + (int)n.size() - 1; }
};

Runs runs_of(const std::vector<int>& q) {
  Runs r;
  if (q.empty()) return r;
  r.q0 = q.front();
  const int span = q.back() - q.front() + 1;
  r.st.assign(span, 0);
  r.n.assign(span, 0);
  for (size_t a = 0; a < q.size(); ++a) {
    const int k = q[a] - r.q0;
    if (r.n[k] == 0) r.st[k] = (int)a;
    ++r.n[k];
  }
  return r;
}

// sigma = (s1, s2, s3) -> index within the sigmas of its total Delta (lexicographic)
struct SigmaTable {
  int d = 0, nDelta = 0;
  std::vector<int> idx, nD, gbo;  // idx[sigma], nD[Delta], gbo[Delta] = offset of the Delta block of a gate
  int gsz = 0;                    // complex elements of one gate's blocks
  explicit SigmaTable(int d_) : d(d_) {
    nDelta = 3 * (d - 1) + 1;
    nD.assign(nDelta, 0);
    idx.assign(d * d * d, 0);
    for (int sg = 0; sg < d * d * d; ++sg) {
      const int t = sg / (d * d) + (sg / d) % d + sg % d;
      idx[sg] = nD[t]++;
    }
    gbo.assign(nDelta, 0);
    for (int t = 0; t < nDelta; ++t) { gbo[t] = gsz; gsz += nD[t] * nD[t]; }
  }
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// bump allocation of byte ranges inside an arena
struct Bump {
  size_t used = 0;
  size_t take(size_t bytes) {
    const size_t o = used;
    used = align256(used + std::max<size_t>(bytes, 16));
    return o;
  }
};

int ensure_arena(tebd_ctx* c, U1Arena& a, size_t bytes) {
  if (a.cap >= bytes) return TEBD_OK;
  if (a.base) {
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail_cuda(c);
    cudaFree(a.base);
  }
  a.base = nullptr;
  a.cap = 0;
  const size_t want = align256(bytes + bytes / 4);  // head-room for the next growth
  if (cudaMalloc(&a.base, want) != cudaSuccess) {
    cudaGetLastError();
    return TEBD_ERR_OOM;
  }
  a.cap = want;
  return TEBD_OK;
}

int grow_ring(tebd_ctx* c, std::vector<void*>& ring, size_t& have, int count, size_t bytes) {
  if (have >= bytes && (int)ring.size() == count) return TEBD_OK;
  if (!ring.empty()) {
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return fail_cuda(c);
    for (void* p : ring) cudaFree(p);
  }
  ring.clear();
  have = 0;
  const size_t want = align256(bytes + bytes / 4);
  for (int i = 0; i < count; ++i) {
    void* p = nullptr;
    if (cudaMalloc(&p, want) != cudaSuccess) {
      cudaGetLastError();
      for (void* q : ring) cudaFree(q);
      ring.clear();
      return TEBD_ERR_OOM;
    }
    ring.push_back(p);
  }
  have = want;
  return TEBD_OK;
}

int ensure_ring(tebd_ctx* c, size_t bytes) { return grow_ring(c, c->u1w->ring, c->u1w->ring_bytes, RING, bytes); }
int ensure_ering(tebd_ctx* c, size_t bytes) { return grow_ring(c, c->u1w->ering, c->u1w->ering_bytes, ERING, bytes); }

int ensure_back(tebd_ctx* c, size_t n) {
  U1Work& w = *c->u1w;
  if (w.h_back_n >= n) return TEBD_OK;
  if (w.h_back) cudaFreeHost(w.h_back);  // only touched after a synchronisation
  w.h_back = nullptr;
  w.h_back_n = 0;
  if (cudaMallocHost(&w.h_back, n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return TEBD_ERR_OOM;
  }
  w.h_back_n = n;
  return TEBD_OK;
}

// Staging of descriptor arrays: host pinned -> device, one region per upload.
// The buffers alternate by chunk; before a buffer is reused, the event recorded
// after its last use (the end of the chunk before last) is waited for.
int stage_begin_chunk(tebd_ctx* c) {
  U1Work& w = *c->u1w;
  w.parity ^= 1;
  w.stage_used = 0;
  if (w.ev[w.parity] && cudaEventSynchronize(w.ev[w.parity]) != cudaSuccess) return fail_cuda(c);
  for (auto& b : w.retired[w.parity]) {
    cudaFreeHost(b.first);
    cudaFree(b.second);
  }
  w.retired[w.parity].clear();
  return TEBD_OK;
}

int stage_end_chunk(tebd_ctx* c) {
  U1Work& w = *c->u1w;
  if (!w.ev[w.parity] && cudaEventCreateWithFlags(&w.ev[w.parity], cudaEventDisableTiming) != cudaSuccess)
    return fail_cuda(c);
  if (cudaEventRecord(w.ev[w.parity], c->stream) != cudaSuccess) return fail_cuda(c);
  return TEBD_OK;
}

// Copy bytes to the device through the current staging buffer; returns the device address.
template <typename T>
T* stage(tebd_ctx* c, const std::vector<T>& v, int* err) {
  U1Work& w = *c->u1w;
  const int p = w.parity;
  const size_t bytes = align256(std::max<size_t>(v.size() * sizeof(T), 16));
  if (w.stage_used + bytes > w.stage_cap[p]) {
    // grow: what was staged earlier in this chunk stays where it is (kernels may still
    // read it), so the old buffers are retired and freed once this parity is next idle
    const size_t want = std::max<size_t>(2 * w.stage_cap[p], align256(bytes) * 4 + (size_t(1) << 20));
    char *h = nullptr, *d = nullptr;
    if (cudaMallocHost(&h, want) != cudaSuccess || cudaMalloc(&d, want) != cudaSuccess) {
      cudaGetLastError();
      if (h) cudaFreeHost(h);
      *err = TEBD_ERR_OOM;
      return nullptr;
    }
    if (w.h_stage[p]) w.retired[p].push_back({w.h_stage[p], w.d_stage[p]});
    w.h_stage[p] = h;
    w.d_stage[p] = d;
    w.stage_cap[p] = want;
    w.stage_used = 0;
  }
  char* hp = w.h_stage[p] + w.stage_used;
  char* dp = w.d_stage[p] + w.stage_used;
  if (!v.empty()) std::memcpy(hp, v.data(), v.size() * sizeof(T));
  if (cudaMemcpyAsync(dp, hp, bytes, cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
    *err = fail_cuda(c);
    return nullptr;
  }
  w.stage_used += bytes;
  return reinterpret_cast<T*>(dp);
}

int launch_moves(tebd_ctx* c, const std::vector<Move>& mv) {
  if (mv.empty()) return TEBD_OK;
  std::vector<long long> ts(mv.size() + 1);
  long long tiles = 0;
  for (size_t i = 0; i < mv.size(); ++i) {
    ts[i] = tiles;
    tiles += ((long long)mv[i].rows * mv[i].cols + MV_TILE - 1) / MV_TILE;
  }
  ts[mv.size()] = tiles;
  if (tiles == 0) return TEBD_OK;
  int err = TEBD_OK;
  Move* dmv = stage(c, mv, &err);
  if (err) return err;
  long long* dts = stage(c, ts, &err);
  if (err) return err;
  k_move<<<(unsigned)tiles, 256, 0, c->stream>>>(dmv, dts, (int)mv.size());
  c->launches += 1;
  return check_launch(c);
}

// Extent checks: every block copy and product the planner emits is checked on the
// host against the allocation it addresses before anything is launched, so a
// planning error is reported as TEBD_ERR_STATE instead of reaching past a buffer.
struct Span {
  const char* lo = nullptr;
  const char* hi = nullptr;
};
Span span_of(const void* p, size_t bytes) {
  return Span{static_cast<const char*>(p), static_cast<const char*>(p) + bytes};
}

// Does the rows x cols block with element (i, j) at p + (i rs + j cs) elements lie inside sp?
bool fits(const void* p, size_t elem, long long rows, long long cols, long long rs, long long cs, const Span& sp) {
  if (rows <= 0 || cols <= 0) return true;
  if (rs < 0 || cs < 0 || !p || !sp.lo) return false;
  const char* first = static_cast<const char*>(p);
  const char* last = first + ((rows - 1) * rs + (cols - 1) * cs) * (long long)elem;
  return first >= sp.lo && last + elem <= sp.hi;
}

struct Checker {
  bool ok = true;
  void need(bool cond, const char* what) {
    if (!cond && ok) std::fprintf(stderr, "ptebd: blocked-update plan out of bounds (%s)\n", what);
    ok = ok && cond;
  }
};

Move gather(Checker& ck, const char* what, const void* sv, long long rs, const Span& ssp, void* pk, long long ldp,
            const Span& psp, int rows, int cols, bool real = false) {
  const size_t e = real ? 8 : 16;
  ck.need(fits(sv, e, rows, cols, rs, 1, ssp) && fits(pk, e, rows, cols, ldp, 1, psp), what);
  return Move{const_cast<void*>(sv), pk, rs, 1, ldp, rows, cols, 0, real ? 1 : 0};
}
Move scatter(Checker& ck, const char* what, void* sv, long long rs, const Span& ssp, const void* pk, long long ldp,
             const Span& psp, int rows, int cols) {
  ck.need(fits(sv, 16, rows, cols, rs, 1, ssp) && fits(pk, 16, rows, cols, ldp, 1, psp), what);
  return Move{sv, const_cast<void*>(pk), rs, 1, ldp, rows, cols, 1, 0};
}

// ---- host: products on the engines of the dense form ----------------------------------
// C (M x N, ldc) = alpha A op(B) [+ C]: A M x K (lda), op(B) = B (K x N, ldb) or B^+ (B stored N x K).
struct Prod {
  const double2* A;
  long long lda;
  const double2* B;
  long long ldb;
  double2* C;
  long long ldc;
  int M, N, K;
  int opB;  // OP_N or OP_C
  double alpha;
  int accumulate;
};

size_t oz_bytes(const Prod& p) { return oz_workspace_bytes(p.M, p.N, p.K, false); }

void check_prod(Checker& ck, const char* what, const Prod& p, const Span& sa, const Span& sb, const Span& sc) {
  ck.need(fits(p.A, 16, p.M, p.K, p.lda, 1, sa), what);
  ck.need(p.opB == OP_C ? fits(p.B, 16, p.N, p.K, p.ldb, 1, sb) : fits(p.B, 16, p.K, p.N, p.ldb, 1, sb), what);
  ck.need(fits(p.C, 16, p.M, p.N, p.ldc, 1, sc), what);
}

// engine: 0 FP64 CUDA cores, 1 split 3xTF32 tensor cores, 2 exact-digit tensor cores
int run_prods(tebd_ctx* c, const std::vector<Prod>& ps, int engine) {
  if (ps.empty()) return TEBD_OK;
  if (engine == 2) {
    size_t need = 0;
    for (const Prod& p : ps) need = std::max(need, oz_bytes(p));
    if (int r = ensure_ring(c, need)) return r;
    std::vector<OzProb> oz;
    for (const Prod& p : ps) {
      OzProb q{};
      q.a = OzOperand{p.A, p.lda, 1, nullptr, 1, 0};
      q.b = p.opB == OP_C ? OzOperand{p.B, p.ldb, 1, nullptr, 1, 1} : OzOperand{p.B, 1, p.ldb, nullptr, 1, 0};
      q.M = p.M; q.N = p.N; q.K = p.K; q.C = p.C; q.ldc = p.ldc; q.alpha = p.alpha; q.beta = p.accumulate;
      q.row_div = q.col_div = 1;
      q.ws = c->u1w->ring[oz.size() % OZ_MAXP];
      oz.push_back(q);
    }
    c->launches += oz_gemm_launch(oz, c->d_status, c->stream);
    return check_launch(c);
  }
  // (an accumulating product is not eligible for the 3xTF32 kernel: Gemm::launch then keeps FP64)
  Gemm gn(true, OP_N, OP_N), gc(true, OP_N, OP_C);
  for (const Prod& p : ps) {
    GemmProb& g = (p.opB == OP_C ? gc : gn).add(p.M, p.N, p.K, p.A, p.lda, p.B, p.ldb, p.C, p.ldc);
    g.alpha_re = p.alpha;
    g.accumulate = p.accumulate;
  }
  const bool tf32 = engine == 1;
  c->launches += gn.launch(c->stream, tf32, c->d_status);
  c->launches += gc.launch(c->stream, tf32, c->d_status);
  return check_launch(c);
}

// The gate products (C = G X, G nd x nd with lda = nd, X and C nd x N with row stride N) in
// one launch per register bucket of nd.
int launch_gate_blocks(tebd_ctx* c, const std::vector<Prod>& ps) {
  constexpr int NB = 4;
  const int cap[NB] = {8, 20, 32, 48};
  std::vector<GateBlk> bk[NB];
  int blocks[NB] = {};
  for (const Prod& p : ps) {
    if (p.M != p.K || p.lda != p.K || p.ldb != p.N || p.ldc != p.N || p.opB != OP_N || p.accumulate ||
        p.alpha != 1.0 || p.M > cap[NB - 1]) {
      std::fprintf(stderr, "ptebd: gate block outside the gate kernel's shapes (nd = %d)\n", p.M);
      return TEBD_ERR_STATE;
    }
    int b = 0;
    while (cap[b] < p.M) ++b;
    const long long nblk = (p.N + 127) / 128;
    if ((long long)blocks[b] + nblk > 2000000000LL) return TEBD_ERR_STATE;
    bk[b].push_back(GateBlk{p.A, p.B, p.C, (long long)p.N, p.M, blocks[b]});
    blocks[b] += (int)nblk;
  }
  for (int b = 0; b < NB; ++b) {
    if (bk[b].empty() || blocks[b] == 0) continue;
    int err = TEBD_OK;
    GateBlk* d = stage(c, bk[b], &err);
    if (err) return err;
    const int n = (int)bk[b].size();
    switch (b) {
      case 0: k_gate_blocks<8><<<blocks[b], 128, 0, c->stream>>>(d, n); break;
      case 1: k_gate_blocks<20><<<blocks[b], 128, 0, c->stream>>>(d, n); break;
      case 2: k_gate_blocks<32><<<blocks[b], 128, 0, c->stream>>>(d, n); break;
      default: k_gate_blocks<48><<<blocks[b], 128, 0, c->stream>>>(d, n); break;
    }
    c->launches += 1;
  }
  return check_launch(c);
}

// ---- host: one cut (SVD) of the blocked update ---------------------------------------------

struct CutBlk {
  int c = 0;             // charge of the cut
  int b = 0, n = 0;      // rows, columns of the packed block
  std::vector<int> rs;   // row start of each row group
  std::vector<int> cs;   // column start of each column group
  int kmax = 0, K = 0;   // eigenvectors possible / computed
  // Gram side: the smaller of (lam P)(lam P)^+ (b x b, left) and (lam P)^+ (lam P) (n x n,
  // right).  Both have the squared singular values as their non-zero eigenvalues; the
  // right one's eigenvectors are the right singular vectors themselves.
  bool right() const { return n < b; }
  int g() const { return right() ? n : b; }
  int cnt = 0, kst = 0;  // kept values, their start on the new bond
  double trace = 0.0;
  size_t oP, oLam, oH, od, oe, oev, otau, op, opart, otr, oZ, oZ2, oS, owork, oU, opan, oY, oV, oW, oSn, oOut;
};

struct Cut {
  std::vector<CutBlk> blk;
  int chi_cap = 1;
  double w_cut = 0.0, eps_rel = 1e-12;  // the owning simulation's options
  double total = 0.0;
  double total_fixed = -1.0;  // if >= 0: ||M||_F^2 of a partial decomposition (rule T's tail)
  size_t oS, oRow, oCnt, oChi, oNorm, oW;  // truncation outputs
  int chi = 1;
  double norm = 1.0, w = 0.0;
};

size_t eig_ws_bytes(int b, int kmax) {
  size_t z = 0;
  auto upd = [&](size_t x) { z = std::max(z, x); };
  upd(oz_workspace_bytes(b, b, 64, false));
  upd(oz_workspace_bytes(64, 64, b, true));
  upd(oz_workspace_bytes(kmax, 64, b, false));
  upd(oz_workspace_bytes(kmax, 64, 64, false));
  upd(oz_workspace_bytes(kmax, b, 64, false));
  upd(oz_workspace_bytes(kmax, kmax, b, true));
  upd(oz_workspace_bytes(b, kmax, kmax, false));
  return z;
}

// arena layout of a cut's blocks (sizes known before the cut is taken)
void layout_cut(Cut& cut, Bump& bp) {
  for (CutBlk& B : cut.blk) {
    const size_t b = B.b, n = B.n, k = B.kmax, g = B.g();  // the eigen-solver works on g x g
    B.oP = bp.take(16 * b * n);
    B.oLam = bp.take(8 * b);
    B.oH = bp.take(16 * g * g);
    B.od = bp.take(8 * g);
    B.oe = bp.take(8 * g);
    B.oev = bp.take(8 * g);
    B.otau = bp.take(16 * g);
    B.op = bp.take(16 * g);
    B.opart = bp.take(16 * (size_t)EIG_PARTS);
    B.otr = bp.take(8);
    B.oZ = bp.take(8 * g * k);
    B.oZ2 = bp.take(8 * g * k);
    B.oS = bp.take(8 * k * k);
    B.owork = bp.take(40 * g * k);
    B.oU = bp.take(16 * k * g);
    B.opan = bp.take(16 * eig_panel_doubles2((int)g));
    B.oY = bp.take(16 * k * n);
    B.oV = bp.take(16 * k * n);
    B.oW = bp.take(16 * k * n);
    B.oSn = bp.take(16 * k * k);
    B.oOut = bp.take(16 * b * k);
  }
  const size_t nb = cut.blk.size();
  size_t ncand = 0;
  for (const CutBlk& B : cut.blk) ncand += B.kmax;
  cut.oS = bp.take(8 * std::max<size_t>(ncand, 1));
  cut.oRow = bp.take(4 * std::max<size_t>(ncand, 1));
  cut.oCnt = bp.take(4 * std::max<size_t>(nb, 1));
  cut.oChi = bp.take(4);
  cut.oNorm = bp.take(8);
  cut.oW = bp.take(8);
}

template <typename T>
T* at(char* base, size_t off) {
  return reinterpret_cast<T*>(base + off);
}

// Gram, eigen-decomposition, projection and truncation of every cut of the batch.
// cuts[t] lives in arena bases[t]; lam_out[t] receives the kept normalised values.
int decompose(tebd_ctx* c, std::vector<Cut*>& cuts, std::vector<char*>& bases, std::vector<double*>& lam_out) {
  const int prec = c->precision;
  const bool mixed = prec >= 1;
  const size_t nc = cuts.size();
  // Gram matrices H_c = (lam P_c)(lam P_c)^+, or (lam P_c)^+ (lam P_c) where that is smaller
  {
    double w = 0.0;
    Gemm g(true, OP_N, OP_C), gr(true, OP_C, OP_N);
    std::vector<OzProb> oz;
    size_t need = 0;
    for (size_t t = 0; t < nc; ++t)
      for (CutBlk& B : cuts[t]->blk) {
        char* a = bases[t];
        if (B.right()) {  // H[i][j] = sum_r lam_r^2 conj(P[r][i]) P[r][j], n x n
          w += 4.0 * (double)B.n * B.n * B.b;
          if (mixed) {
            need = std::max(need, oz_workspace_bytes(B.n, B.n, B.b, true));
            OzProb q{};
            q.a = OzOperand{at<double2>(a, B.oP), 1, B.n, at<double>(a, B.oLam), 1, 1};
            q.M = q.N = B.n; q.K = B.b; q.C = at<double2>(a, B.oH); q.ldc = B.n; q.alpha = 1.0;
            q.row_div = q.col_div = 1;
            q.herm = q.gram = 1;
            oz.push_back(q);
          } else {
            GemmProb& p = gr.add(B.n, B.n, B.b, at<double2>(a, B.oP), B.n, at<double2>(a, B.oP), B.n,
                                 at<double2>(a, B.oH), B.n);
            p.s_red = p.s_red_b = at<double>(a, B.oLam);
            p.herm = 1;
          }
          continue;
        }
        w += 4.0 * (double)B.b * B.b * B.n;
        if (mixed) {
          need = std::max(need, oz_workspace_bytes(B.b, B.b, B.n, true));
          OzProb q{};
          q.a = OzOperand{at<double2>(a, B.oP), B.n, 1, nullptr, 1, 0};
          q.M = q.N = B.b; q.K = B.n; q.C = at<double2>(a, B.oH); q.ldc = B.b; q.alpha = 1.0;
          q.s_row = q.s_col = at<double>(a, B.oLam);
          q.row_div = q.col_div = 1;
          q.herm = q.gram = 1;
          oz.push_back(q);
        } else {
          GemmProb& p = g.add(B.b, B.b, B.n, at<double2>(a, B.oP), B.n, at<double2>(a, B.oP), B.n,
                              at<double2>(a, B.oH), B.b);
          p.s_row = p.s_col = at<double>(a, B.oLam);
          p.herm = 1;
        }
      }
    ProfScope ps(c, TEBD_PROF_GRAM, w);
    if (mixed) {
      if (int r = ensure_ring(c, need)) return r;
      for (size_t j = 0; j < oz.size(); ++j) oz[j].ws = c->u1w->ring[j % OZ_MAXP];
      c->launches += oz_gemm_launch(oz, c->d_status, c->stream);
    } else {
      c->launches += g.launch(c->stream);
      c->launches += gr.launch(c->stream);
    }
    if (int r = check_launch(c)) return r;
  }
  // eigen-decomposition of every block, in batches of similar size
  struct Job { size_t t; CutBlk* B; };
  std::vector<Job> jobs;
  size_t ews = 0;
  for (size_t t = 0; t < nc; ++t)
    for (CutBlk& B : cuts[t]->blk) {
      jobs.push_back({t, &B});
      if (mixed) ews = std::max(ews, eig_ws_bytes(B.g(), B.kmax));
    }
  std::stable_sort(jobs.begin(), jobs.end(), [](const Job& x, const Job& y) { return x.B->g() > y.B->g(); });
  if (mixed)
    if (int r = ensure_ering(c, ews)) return r;
  auto mat = [&](const Job& j) {
    char* a = bases[j.t];
    CutBlk& B = *j.B;
    EigMat M{};
    M.H = at<double2>(a, B.oH); M.d = at<double>(a, B.od); M.e = at<double>(a, B.oe);
    M.tau = at<double2>(a, B.otau); M.part = at<double2>(a, B.opart); M.p = at<double2>(a, B.op);
    M.evals = at<double>(a, B.oev); M.trace = at<double>(a, B.otr); M.Z = at<double>(a, B.oZ);
    M.Z2 = at<double>(a, B.oZ2); M.S = at<double>(a, B.oS); M.work = at<double>(a, B.owork);
    M.U = at<double2>(a, B.oU); M.pan = at<double2>(a, B.opan);
    M.m = B.g(); M.kmax = B.kmax; M.K = B.K;
    return M;
  };
  void* ozw[EIG_MAXP] = {};
  if (mixed)
    for (int i = 0; i < EIG_MAXP; ++i) ozw[i] = c->u1w->ering[i];
  {
    double w = 0.0;
    for (const Job& j : jobs) w += 16.0 / 3.0 * std::pow((double)j.B->g(), 3);
    ProfScope ps(c, TEBD_PROF_TRIDIAG, w);
    for (size_t g0 = 0; g0 < jobs.size(); g0 += EIG_MAXP) {
      EigBatch eb{};
      eb.bar = c->d_bar;
      eb.wait_clocks = c->wait_clocks;
      eb.panel_blocks = c->panel_blocks;
      for (size_t j = g0; j < std::min(jobs.size(), g0 + EIG_MAXP); ++j) eb.a[eb.n++] = mat(jobs[j]);
      c->launches += eig_trace(eb, c->stream);
      const int nl = eig_tridiagonalize(eb, mixed, ozw, c->d_status, c->stream);
      if (nl < 0) {
        cudaGetLastError();
        std::fprintf(stderr, "ptebd: cooperative launch of the tridiagonal reduction refused\n");
        return fail_cuda(c);
      }
      c->launches += nl;
    }
  }
  {
    ProfScope ps(c, TEBD_PROF_BISECT, 0.0);
    // eigenvalues needed per block: at most the cut's chi_cap largest, above the floor
    std::vector<EigMat> em;
    std::vector<ThrCut> tcut(nc);
    std::vector<CutBlk*> order;
    for (size_t t = 0; t < nc; ++t) {
      tcut[t].n = (int)cuts[t]->blk.size();
      tcut[t].target = cuts[t]->chi_cap;
      tcut[t].floor_rel = std::max(0.01 * cuts[t]->eps_rel, 1e-15);
      for (CutBlk& B : cuts[t]->blk) {
        em.push_back(mat(Job{t, &B}));
        order.push_back(&B);
      }
    }
    U1Work& w = *c->u1w;
    if (w.d_counts_n < em.size()) {
      if (w.d_counts) cudaFree(w.d_counts);  // idle: only used between the synchronisations below
      w.d_counts = nullptr;
      w.d_counts_n = 0;
      if (cudaMalloc(&w.d_counts, sizeof(int) * std::max<size_t>(em.size(), 64) * 2) != cudaSuccess) {
        cudaGetLastError();
        return TEBD_ERR_OOM;
      }
      w.d_counts_n = std::max<size_t>(em.size(), 64) * 2;
    }
    int err = TEBD_OK;
    EigMat* dem = stage(c, em, &err);
    if (err) return err;
    size_t off = 0;
    for (size_t t = 0; t < nc; ++t) {
      tcut[t].mats = dem + off;
      tcut[t].kmax_out = w.d_counts + off;
      off += tcut[t].n;
    }
    ThrCut* dtc = stage(c, tcut, &err);
    if (err) return err;
    c->launches += eig_cut_counts(dtc, (int)nc, c->stream);
    if (int r = ensure_back(c, em.size() / 2 + 8)) return r;
    if (cudaMemcpyAsync(c->u1w->h_back, w.d_counts, sizeof(int) * em.size(), cudaMemcpyDeviceToHost, c->stream) !=
        cudaSuccess)
      return fail_cuda(c);
    if (int r = sync(c)) return r;
    const int* cnt = reinterpret_cast<const int*>(c->u1w->h_back);
    for (size_t i = 0; i < order.size(); ++i) order[i]->kmax = std::max(0, std::min(order[i]->kmax, cnt[i]));
    std::vector<Job> bj;
    for (const Job& j : jobs)
      if (j.B->kmax > 0) bj.push_back(j);
    for (size_t g0 = 0; g0 < bj.size(); g0 += EIG_MAXP) {
      EigBatch eb{};
      for (size_t j = g0; j < std::min(bj.size(), g0 + EIG_MAXP); ++j) eb.a[eb.n++] = mat(bj[j]);
      c->launches += eig_bisect(eb, c->stream);
    }
  }
  if (int r = check_launch(c)) return r;
  // read back eigenvalues and traces
  size_t nback = 2;
  for (const Job& j : jobs) nback += j.B->kmax + 1;
  if (int r = ensure_back(c, nback)) return r;
  double* hb = c->u1w->h_back;
  {
    size_t o = 0;
    for (const Job& j : jobs) {
      char* a = bases[j.t];
      cudaMemcpyAsync(hb + o, at<double>(a, j.B->oev), 8 * j.B->kmax, cudaMemcpyDeviceToHost, c->stream);
      cudaMemcpyAsync(hb + o + j.B->kmax, at<double>(a, j.B->otr), 8, cudaMemcpyDeviceToHost, c->stream);
      o += j.B->kmax + 1;
    }
    cudaMemcpyAsync(hb + o, c->d_bar + 2, sizeof(unsigned int), cudaMemcpyDeviceToHost, c->stream);
    if (int r = sync(c)) return r;
    if (*reinterpret_cast<unsigned int*>(hb + o) != 0) {
      c->sticky = TEBD_ERR_TIMEOUT;
      return TEBD_ERR_TIMEOUT;
    }
  }
  std::vector<double> ev0(jobs.size());
  {
    size_t o = 0;
    for (auto& cut : cuts) cut->total = 0.0;
    for (size_t q = 0; q < jobs.size(); ++q) {
      Job& j = jobs[q];
      j.B->trace = hb[o + j.B->kmax];
      if (!is_fin(j.B->trace)) {
        c->sticky = TEBD_ERR_NONFINITE;
        return TEBD_ERR_NONFINITE;
      }
      cuts[j.t]->total += j.B->trace;
      o += j.B->kmax + 1;
    }
    for (auto& cut : cuts)
      if (cut->total_fixed >= 0.0) cut->total = cut->total_fixed;
    o = 0;
    for (size_t q = 0; q < jobs.size(); ++q) {
      Job& j = jobs[q];
      const double total = cuts[j.t]->total;
      if (!(total > 0.0) || !is_fin(total)) {
        c->sticky = TEBD_ERR_NONFINITE;
        return TEBD_ERR_NONFINITE;
      }
      // vectors for every eigenvalue that could pass the eps_rel floor (100x margin), as in the dense form
      const double floor_v = std::max(0.01 * cuts[j.t]->eps_rel, 1e-15) * total;
      const double* ev = hb + o;
      int K = 0;
      while (K < j.B->kmax && ev[K] > floor_v) ++K;
      j.B->K = K;
      ev0[q] = j.B->kmax > 0 ? ev[0] : -1.0;
      o += j.B->kmax + 1;
    }
    // As in the dense form, vectors only for the chi_cap largest eigenvalues of the cut
    // (merged over its blocks; every value equal to the chi_cap-th is kept too): rule T
    // keeps at most chi_cap values, so the others would be computed and dropped.
    {
      std::vector<std::vector<double>> cand(nc);
      size_t o2 = 0;
      for (size_t q = 0; q < jobs.size(); ++q) {
        const Job& j = jobs[q];
        for (int k = 0; k < j.B->K; ++k) cand[j.t].push_back(hb[o2 + k]);
        o2 += j.B->kmax + 1;
      }
      std::vector<double> thr(nc, -1.0);
      for (size_t t = 0; t < nc; ++t) {
        auto& v = cand[t];
        const size_t cap = (size_t)cuts[t]->chi_cap;
        if (v.size() > cap) {
          std::nth_element(v.begin(), v.begin() + (cap - 1), v.end(), std::greater<double>());
          thr[t] = v[cap - 1];
        }
      }
      o2 = 0;
      for (size_t q = 0; q < jobs.size(); ++q) {
        Job& j = jobs[q];
        if (thr[j.t] >= 0.0) {
          const double* ev = hb + o2;
          int K = 0;
          while (K < j.B->K && ev[K] >= thr[j.t]) ++K;
          j.B->K = K;
        }
        o2 += j.B->kmax + 1;
      }
    }
    // every cut keeps at least one value: its block with the largest eigenvalue
    for (size_t t = 0; t < nc; ++t) {
      int best = -1, any = 0;
      for (size_t q = 0; q < jobs.size(); ++q)
        if (jobs[q].t == t) {
          any += jobs[q].B->K;
          if (best < 0 || ev0[q] > ev0[best]) best = (int)q;
        }
      if (any == 0 && best >= 0) jobs[best].B->K = 1;
    }
  }
  // eigenvectors of the blocks that keep any
  {
    std::vector<Job> vj;
    double w = 0.0;
    for (const Job& j : jobs)
      if (j.B->K > 0) {
        vj.push_back(j);
        w += 8.0 * (double)j.B->g() * j.B->g() * j.B->K + 12.0 * (double)j.B->g() * j.B->K * j.B->K;
      }
    ProfScope ps(c, TEBD_PROF_EIGVEC, w);
    for (size_t g0 = 0; g0 < vj.size(); g0 += EIG_MAXP) {
      EigBatch eb{};
      eb.bar = c->d_bar;
      eb.wait_clocks = c->wait_clocks;
      eb.panel_blocks = c->panel_blocks;
      for (size_t j = g0; j < std::min(vj.size(), g0 + EIG_MAXP); ++j) eb.a[eb.n++] = mat(vj[j]);
      c->launches += eig_vectors(eb, mixed, ozw, c->d_status, c->stream);
    }
    if (int r = check_launch(c)) return r;
  }
  // projection Y_c = U_c^+ (lam P_c); for a right Gram Y_c = diag(s) Z_c^+ (k_right_*)
  {
    double w = 0.0;
    Gemm g(true, OP_CJ, OP_N), gt(true, OP_N, OP_C);
    std::vector<OzProb> oz;
    std::vector<RightRows> rr;
    int rmaxK = 0;
    size_t need = 0;
    for (size_t t = 0; t < nc; ++t)
      for (CutBlk& B : cuts[t]->blk) {
        if (B.K == 0) continue;
        char* a = bases[t];
        w += 8.0 * (double)B.K * B.b * B.n;
        if (B.right()) {  // T = (lam P) Y^+ with Y = conj(Z), into the rebuild's (not yet used) buffer
          rr.push_back(RightRows{at<double2>(a, B.oU), at<double2>(a, B.oY), at<double2>(a, B.oOut), B.K, B.n, B.b});
          rmaxK = std::max(rmaxK, B.K);
          if (mixed) {
            need = std::max(need, oz_workspace_bytes(B.b, B.K, B.n, false));
            OzProb q{};
            q.a = OzOperand{at<double2>(a, B.oP), B.n, 1, nullptr, 1, 0};
            q.b = OzOperand{at<double2>(a, B.oY), B.n, 1, nullptr, 1, 1};
            q.M = B.b; q.N = B.K; q.K = B.n; q.C = at<double2>(a, B.oOut); q.ldc = B.K; q.alpha = 1.0;
            q.s_row = at<double>(a, B.oLam);
            q.row_div = q.col_div = 1;
            oz.push_back(q);
          } else {
            GemmProb& p = gt.add(B.b, B.K, B.n, at<double2>(a, B.oP), B.n, at<double2>(a, B.oY), B.n,
                                 at<double2>(a, B.oOut), B.K);
            p.s_row = at<double>(a, B.oLam);
          }
          continue;
        }
        if (mixed) {
          need = std::max(need, oz_workspace_bytes(B.K, B.n, B.b, false));
          OzProb q{};
          q.a = OzOperand{at<double2>(a, B.oU), B.b, 1, at<double>(a, B.oLam), 1, 1};
          q.b = OzOperand{at<double2>(a, B.oP), 1, B.n, nullptr, 1, 0};
          q.M = B.K; q.N = B.n; q.K = B.b; q.C = at<double2>(a, B.oY); q.ldc = B.n; q.alpha = 1.0;
          q.row_div = q.col_div = 1;
          oz.push_back(q);
        } else {
          GemmProb& p = g.add(B.K, B.n, B.b, at<double2>(a, B.oU), B.b, at<double2>(a, B.oP), B.n,
                              at<double2>(a, B.oY), B.n);
          p.s_red = at<double>(a, B.oLam);
          p.red_div = 1;
        }
      }
    ProfScope ps(c, TEBD_PROF_PROJECT, w);
    RightRows* drr = nullptr;
    if (!rr.empty()) {
      int err = TEBD_OK;
      drr = stage(c, rr, &err);
      if (err) return err;
      for (size_t y0 = 0; y0 < rr.size(); y0 += 65535) {
        const unsigned ny = (unsigned)std::min<size_t>(65535, rr.size() - y0);
        k_right_conj<<<dim3((unsigned)rmaxK, ny), 128, 0, c->stream>>>(drr + y0);
        c->launches += 1;
      }
    }
    if (mixed) {
      if (int r = ensure_ring(c, need)) return r;
      for (size_t j = 0; j < oz.size(); ++j) oz[j].ws = c->u1w->ring[j % OZ_MAXP];
      c->launches += oz_gemm_launch(oz, c->d_status, c->stream);
    } else {
      c->launches += g.launch(c->stream);
      c->launches += gt.launch(c->stream);
    }
    for (size_t y0 = 0; y0 < rr.size(); y0 += 65535) {
      const unsigned ny = (unsigned)std::min<size_t>(65535, rr.size() - y0);
      k_right_scale<<<dim3((unsigned)rmaxK, ny), 128, 0, c->stream>>>(drr + y0);
      c->launches += 1;
    }
    if (int r = check_launch(c)) return r;
  }
  // rule T on the merged spectrum of each cut
  {
    ProfScope ps(c, TEBD_PROF_TRUNCATE, 0.0);
    std::vector<TruncCut> tc(nc);
    std::vector<TruncBlk> allb;
    std::vector<size_t> boff(nc);
    int maxP = 1;
    for (size_t t = 0; t < nc; ++t) {
      Cut& cut = *cuts[t];
      boff[t] = allb.size();
      int ncand = 0;
      for (CutBlk& B : cut.blk) {
        allb.push_back(TruncBlk{at<double2>(bases[t], B.oY), B.K, B.n});
        ncand += B.K;
      }
      if (cut.blk.size() > 1024 || ncand > 16384) {
        std::fprintf(stderr, "ptebd: a cut with %zu charge blocks and %d candidates exceeds the blocked truncation\n",
                     cut.blk.size(), ncand);
        c->sticky = TEBD_ERR_ARG;
        return TEBD_ERR_ARG;
      }
      int P = 1;
      while (P < ncand) P <<= 1;
      maxP = std::max(maxP, P);
    }
    int err = TEBD_OK;
    TruncBlk* dallb = stage(c, allb, &err);
    if (err) return err;
    for (size_t t = 0; t < nc; ++t) {
      Cut& cut = *cuts[t];
      char* a = bases[t];
      TruncCut& T = tc[t];
      T.blk = dallb + boff[t];
      T.nb = (int)cut.blk.size();
      T.ncand = 0;
      for (CutBlk& B : cut.blk) T.ncand += B.K;
      T.total = cut.total;
      T.chi_max = cut.chi_cap;
      T.w_cut = cut.w_cut;
      T.eps_rel = cut.eps_rel;
      T.lam_out = lam_out[t];
      T.s_out = at<double>(a, cut.oS);
      T.row_out = at<int>(a, cut.oRow);
      T.counts = at<int>(a, cut.oCnt);
      T.chi_out = at<int>(a, cut.oChi);
      T.norm_out = at<double>(a, cut.oNorm);
      T.w_out = at<double>(a, cut.oW);
      T.status = c->d_status;
    }
    TruncCut* dtc = stage(c, tc, &err);
    if (err) return err;
    const size_t smem = (size_t)maxP * (sizeof(double) + sizeof(int));
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_trunc_u1, cudaFuncAttributeMaxDynamicSharedMemorySize, 16384 * 12);
      attr = true;
    }
    k_trunc_u1<<<(unsigned)nc, TR_THREADS, smem, c->stream>>>(dtc);
    c->launches += 1;
    if (int r = check_launch(c)) return r;
  }
  // read back chi', norms, weights, per-block counts and the status
  size_t nback2 = 4;
  for (size_t t = 0; t < nc; ++t) nback2 += 3 + cuts[t]->blk.size();
  if (int r = ensure_back(c, nback2)) return r;
  hb = c->u1w->h_back;
  {
    size_t o = 0;
    for (size_t t = 0; t < nc; ++t) {
      Cut& cut = *cuts[t];
      char* a = bases[t];
      cudaMemcpyAsync(hb + o, at<double>(a, cut.oNorm), 8, cudaMemcpyDeviceToHost, c->stream);
      cudaMemcpyAsync(hb + o + 1, at<double>(a, cut.oW), 8, cudaMemcpyDeviceToHost, c->stream);
      cudaMemcpyAsync(hb + o + 2, at<int>(a, cut.oChi), 4, cudaMemcpyDeviceToHost, c->stream);
      // counts as ints, two per double slot
      cudaMemcpyAsync(hb + o + 3, at<int>(a, cut.oCnt), 4 * cut.blk.size(), cudaMemcpyDeviceToHost, c->stream);
      o += 3 + cut.blk.size();
    }
    cudaMemcpyAsync(hb + o, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (int r = sync(c)) return r;
    const int st = *reinterpret_cast<const int*>(hb + o);
    if (st != 0) {
      c->sticky = st;
      return st;
    }
    o = 0;
    for (size_t t = 0; t < nc; ++t) {
      Cut& cut = *cuts[t];
      cut.norm = hb[o];
      cut.w = hb[o + 1];
      cut.chi = *reinterpret_cast<const int*>(hb + o + 2);
      const int* cnt = reinterpret_cast<const int*>(hb + o + 3);
      int kst = 0;
      for (size_t b = 0; b < cut.blk.size(); ++b) {
        cut.blk[b].cnt = cnt[b];
        cut.blk[b].kst = kst;
        kst += cnt[b];
        if (cnt[b] < 0 || cnt[b] > cut.blk[b].K) {
          c->sticky = TEBD_ERR_STATE;
          return TEBD_ERR_STATE;
        }
      }
      if (cut.chi < 1 || cut.chi > cut.chi_cap || kst != cut.chi || !is_fin(cut.norm) || !(cut.norm > 0.0)) {
        c->sticky = TEBD_ERR_STATE;
        return TEBD_ERR_STATE;
      }
      o += 3 + cut.blk.size();
    }
  }
  return TEBD_OK;
}

// Kept right vectors of every block: V = kept rows of Y / s, then one Newton-Schulz
// step W = 1.5 V - 0.5 (V V^+) V (W starts as 1.5 V).
int kept_vectors(tebd_ctx* c, std::vector<Cut*>& cuts, std::vector<char*>& bases) {
  std::vector<KeptGather> kg;
  int maxcnt = 0;
  for (size_t t = 0; t < cuts.size(); ++t)
    for (CutBlk& B : cuts[t]->blk) {
      if (B.cnt == 0) continue;
      char* a = bases[t];
      kg.push_back(KeptGather{at<double2>(a, B.oY), at<double2>(a, B.oV), at<double2>(a, B.oW),
                              at<int>(a, cuts[t]->oRow), at<double>(a, cuts[t]->oS), B.n, B.kst, B.cnt});
      maxcnt = std::max(maxcnt, B.cnt);
    }
  if (kg.empty()) return TEBD_OK;
  {
    ProfScope ps(c, TEBD_PROF_TRUNCATE, 0.0);
    int err = TEBD_OK;
    KeptGather* dkg = stage(c, kg, &err);
    if (err) return err;
    for (size_t y0 = 0; y0 < kg.size(); y0 += 65535) {
      const unsigned ny = (unsigned)std::min<size_t>(65535, kg.size() - y0);
      k_kept_gather<<<dim3((unsigned)maxcnt, ny), 128, 0, c->stream>>>(dkg + y0);
      c->launches += 1;
    }
    if (int r = check_launch(c)) return r;
  }
  const bool mixed = c->precision >= 1;
  double w = 0.0;
  std::vector<Prod> gram, app;
  for (size_t t = 0; t < cuts.size(); ++t)
    for (CutBlk& B : cuts[t]->blk) {
      if (B.cnt == 0) continue;
      char* a = bases[t];
      w += 12.0 * (double)B.cnt * B.cnt * B.n;
      gram.push_back(Prod{at<double2>(a, B.oV), B.n, at<double2>(a, B.oV), B.n, at<double2>(a, B.oSn), B.cnt, B.cnt,
                          B.cnt, B.n, OP_C, 1.0, 0});
      app.push_back(Prod{at<double2>(a, B.oSn), B.cnt, at<double2>(a, B.oV), B.n, at<double2>(a, B.oW), B.n, B.cnt,
                         B.n, B.cnt, OP_N, -0.5, 1});
    }
  ProfScope ps(c, TEBD_PROF_PROJECT, w);
  if (int r = run_prods(c, gram, mixed ? 2 : 0)) return r;
  return run_prods(c, app, mixed ? 2 : 0);
}

}  // namespace

// ---- the blocked local update of a batch of triples -----------------------------------------

namespace {

Span site_span(const tebd_ctx* o, int k) { return span_of(o->B[k], 16 * (size_t)o->cap[k] * o->d * o->cap[k + 1]); }
Span lam_span(const tebd_ctx* o, int k) { return span_of(o->lam[k], 8 * (size_t)o->cap[k]); }
Span arena_span(const U1Arena& a) { return span_of(a.base, a.cap); }

int update_chunk_u1_body(tebd_ctx* c, std::vector<Triple>& ts, int tidx) {
  cudaStream_t s = c->stream;
  const int prec = c->precision;
  // engines: contractions (theta, gate, rebuilds) and the gate product
  // engines of the contractions (theta~, rebuilds): FP64, split 3xTF32 or exact digits.
  // The gate product runs on the FP64 CUDA cores in every precision: in the blocked
  // form its reduction is one occupation block (K = n_Delta <= 19, a single tensor-core
  // k-step), where the accumulator's round-towards-zero is not averaged over k-steps;
  // in 3xTF32 it tripled the mixed path's observable error (1.3e-5 against 4.1e-6 at
  // L = 8, t = 1), for about 1 % of the contraction work.
  const int e_con = prec == 1 ? 1 : (prec == 2 ? 2 : 0);
  const size_t nt = ts.size();
  struct Plan {
    // stage A: X_c = B_i B_{i+1} for each charge c of bond i+1
    struct XB { int c, rows, cols, K; std::vector<int> rs, cs; size_t oX, oA, oB; };
    struct TB { int c, rows, cols, K; std::vector<int> rs, cs; size_t oXB, oB2, oT; };
    std::vector<XB> xb;
    std::vector<TB> tb;
    std::vector<long long> NDl, tD;            // per Delta: columns, start in the compact theta
    std::vector<std::vector<long long>> cb;    // cb[Delta][alpha - qlo_l]: column base of (alpha, alpha + Delta)
    long long theta_n = 0;
    size_t oTh, oC, xsize, xoff;
    Cut cut1, cut2;
    Runs rl, r1, r2, rr, r1n;
  };
  std::vector<Plan> pl(nt);
  Checker ck;
  // the local dimension of each triple is its own simulation's (a batch may mix them)
  std::vector<SigmaTable> sgs;
  for (int dd = 0; dd <= 8; ++dd) sgs.emplace_back(std::max(dd, 1));
  // ---- plan the products and the first cut (sizes from the bond charges)
  for (size_t t = 0; t < nt; ++t) {
    Triple& T = ts[t];
    [[maybe_unused]] const int d = T.h->d;
    [[maybe_unused]] const SigmaTable& sg = sgs[d];
    tebd_ctx* o = T.h;
    Plan& P = pl[t];
    T.chl = o->chi[T.i]; T.c1 = o->chi[T.i + 1]; T.c2 = o->chi[T.i + 2]; T.chr = o->chi[T.i + 3];
    P.rl = runs_of(o->q[T.i]); P.r1 = runs_of(o->q[T.i + 1]); P.r2 = runs_of(o->q[T.i + 2]); P.rr = runs_of(o->q[T.i + 3]);
    Bump bp;
    // stage A blocks: charge c of bond i+1 (rows (s1, a), columns (s2, c2))
    const int cA0 = P.rl.lo(), cA1 = P.rl.hi() + d - 1;
    P.xsize = 0;
    for (int cq = cA0; cq <= cA1; ++cq) {
      Plan::XB X{};
      X.c = cq;
      X.rs.assign(d, 0);
      X.cs.assign(d, 0);
      for (int s1 = 0; s1 < d; ++s1) { X.rs[s1] = X.rows; X.rows += P.rl.count(cq - s1); }
      for (int s2 = 0; s2 < d; ++s2) { X.cs[s2] = X.cols; X.cols += P.r2.count(cq + s2); }
      X.K = P.r1.count(cq);
      if (X.rows == 0 || X.cols == 0) continue;
      X.oX = P.xsize;  // X blocks are contiguous so one memset zeroes them all
      P.xsize += 16 * (size_t)X.rows * X.cols;
      P.xb.push_back(X);
    }
    P.xoff = bp.take(P.xsize);
    for (auto& X : P.xb) {
      X.oX += P.xoff;
      X.oA = bp.take(16 * (size_t)X.rows * std::max(X.K, 1));
      X.oB = bp.take(16 * (size_t)std::max(X.K, 1) * X.cols);
    }
    // compact theta~ and C: per Delta, columns over alpha of (a, b) pairs
    const int nDel = sg.nDelta;
    P.NDl.assign(nDel, 0);
    P.tD.assign(nDel, 0);
    P.cb.assign(nDel, std::vector<long long>(P.rl.n.size(), -1));
    for (int dl = 0; dl < nDel; ++dl) {
      for (int al = P.rl.lo(); al <= P.rl.hi(); ++al) {
        const long long na = P.rl.count(al), nb_ = P.rr.count(al + dl);
        if (na == 0 || nb_ == 0) continue;
        P.cb[dl][al - P.rl.lo()] = P.NDl[dl];
        P.NDl[dl] += na * nb_;
      }
      P.tD[dl] = P.theta_n;
      P.theta_n += (long long)sg.nD[dl] * P.NDl[dl];
    }
    P.oTh = bp.take(16 * (size_t)std::max<long long>(P.theta_n, 1));
    P.oC = bp.take(16 * (size_t)std::max<long long>(P.theta_n, 1));
    // stage B blocks: charge c' of bond i+2 (rows (s1, s2, a), columns (s3, b))
    for (int cq = P.r2.lo(); cq <= P.r2.hi(); ++cq) {
      Plan::TB X{};
      X.c = cq;
      X.K = P.r2.count(cq);
      if (X.K == 0) continue;
      X.rs.assign(d * d, 0);
      X.cs.assign(d, 0);
      for (int s1 = 0; s1 < d; ++s1)
        for (int s2 = 0; s2 < d; ++s2) { X.rs[s1 * d + s2] = X.rows; X.rows += P.rl.count(cq - s1 - s2); }
      for (int s3 = 0; s3 < d; ++s3) { X.cs[s3] = X.cols; X.cols += P.rr.count(cq + s3); }
      if (X.rows == 0 || X.cols == 0) continue;
      X.oXB = bp.take(16 * (size_t)X.rows * X.K);
      X.oB2 = bp.take(16 * (size_t)X.K * X.cols);
      X.oT = bp.take(16 * (size_t)X.rows * X.cols);
      P.tb.push_back(X);
    }
    // first cut: charge c after site i (rows (s1, a), columns ((s2, s3), b))
    P.cut1.chi_cap = std::min(o->chi_max, o->cap[T.i + 1]);
    P.cut1.w_cut = o->w_cut;
    P.cut1.eps_rel = o->eps_rel;
    for (int cq = P.rl.lo(); cq <= P.rl.hi() + d - 1; ++cq) {
      CutBlk B{};
      B.c = cq;
      B.rs.assign(d, 0);
      B.cs.assign(d * d, 0);
      for (int s1 = 0; s1 < d; ++s1) { B.rs[s1] = B.b; B.b += P.rl.count(cq - s1); }
      for (int s2 = 0; s2 < d; ++s2)
        for (int s3 = 0; s3 < d; ++s3) { B.cs[s2 * d + s3] = B.n; B.n += P.rr.count(cq + s2 + s3); }
      if (B.b == 0 || B.n == 0) continue;
      B.kmax = std::min({B.b, B.n, P.cut1.chi_cap});
      P.cut1.blk.push_back(B);
    }
    layout_cut(P.cut1, bp);
    if (int r = ensure_arena(c, T.h->u1w->slots[T.slot].a1, bp.used)) return r;
  }
  // ---- stage A: X = B_i B_{i+1}
  {
    std::vector<Move> mv;
    std::vector<Prod> pr;
    double wc = 0.0;
    for (size_t t = 0; t < nt; ++t) {
      Triple& T = ts[t];
      [[maybe_unused]] const int d = T.h->d;
      [[maybe_unused]] const SigmaTable& sg = sgs[d];
      tebd_ctx* o = T.h;
      Plan& P = pl[t];
      char* a = T.h->u1w->slots[T.slot].a1.base;
      const Span sa = arena_span(T.h->u1w->slots[T.slot].a1);
      if (P.xsize && cudaMemsetAsync(a + P.xoff, 0, P.xsize, s) != cudaSuccess) return fail_cuda(c);
      for (auto& X : P.xb) {
        if (X.K == 0) continue;
        const int K = X.K, k0 = P.r1.start(X.c);
        for (int s1 = 0; s1 < d; ++s1) {
          const int n = P.rl.count(X.c - s1);
          if (n == 0) continue;
          const long long base = ((long long)P.rl.start(X.c - s1) * d + s1) * T.c1 + k0;
          mv.push_back(gather(ck, "A: B_i", o->B[T.i] + base, (long long)d * T.c1, site_span(o, T.i),
                              at<double2>(a, X.oA) + (size_t)X.rs[s1] * K, K, sa, n, K));
        }
        for (int s2 = 0; s2 < d; ++s2) {
          const int n = P.r2.count(X.c + s2);
          if (n == 0) continue;
          const long long base = ((long long)k0 * d + s2) * T.c2 + P.r2.start(X.c + s2);
          mv.push_back(gather(ck, "A: B_i+1", o->B[T.i + 1] + base, (long long)d * T.c2, site_span(o, T.i + 1),
                              at<double2>(a, X.oB) + X.cs[s2], X.cols, sa, K, n));
        }
        pr.push_back(Prod{at<double2>(a, X.oA), K, at<double2>(a, X.oB), X.cols, at<double2>(a, X.oX), X.cols, X.rows,
                          X.cols, K, OP_N, 1.0, 0});
        check_prod(ck, "A: product", pr.back(), sa, sa, sa);
        wc += 8.0 * (double)X.rows * X.cols * K;
      }
    }
    if (!ck.ok) return TEBD_ERR_STATE;
    ProfScope ps(c, TEBD_PROF_CONTRACT, wc);
    if (int r = launch_moves(c, mv)) return r;
    if (int r = run_prods(c, pr, e_con)) return r;
  }
  // ---- stage B: theta~ = X B_{i+2}, scattered into the compact layout
  {
    std::vector<Move> mv, sc;
    std::vector<Prod> pr;
    double wc = 0.0;
    for (size_t t = 0; t < nt; ++t) {
      Triple& T = ts[t];
      [[maybe_unused]] const int d = T.h->d;
      [[maybe_unused]] const SigmaTable& sg = sgs[d];
      tebd_ctx* o = T.h;
      Plan& P = pl[t];
      char* a = T.h->u1w->slots[T.slot].a1.base;
      const Span sa = arena_span(T.h->u1w->slots[T.slot].a1);
      if (cudaMemsetAsync(a + P.oTh, 0, 16 * (size_t)std::max<long long>(P.theta_n, 1), s) != cudaSuccess)
        return fail_cuda(c);
      // X block of charge cq, by charge
      auto xfind = [&](int cq) -> const Plan::XB* {
        for (auto& X : P.xb)
          if (X.c == cq) return &X;
        return nullptr;
      };
      for (auto& X : P.tb) {
        const int K = X.K, k0 = P.r2.start(X.c);
        for (int s1 = 0; s1 < d; ++s1)
          for (int s2 = 0; s2 < d; ++s2) {
            const int n = P.rl.count(X.c - s1 - s2);
            if (n == 0) continue;
            const Plan::XB* xs = xfind(X.c - s2);
            if (!xs) return TEBD_ERR_STATE;  // cannot happen: the rows and columns exist
            const double2* src = at<double2>(a, xs->oX) + (size_t)xs->rs[s1] * xs->cols + xs->cs[s2];
            mv.push_back(gather(ck, "B: X", src, xs->cols, sa, at<double2>(a, X.oXB) + (size_t)X.rs[s1 * d + s2] * K, K,
                                sa, n, K));
          }
        for (int s3 = 0; s3 < d; ++s3) {
          const int n = P.rr.count(X.c + s3);
          if (n == 0) continue;
          const long long base = ((long long)k0 * d + s3) * T.chr + P.rr.start(X.c + s3);
          mv.push_back(gather(ck, "B: B_i+2", o->B[T.i + 2] + base, (long long)d * T.chr, site_span(o, T.i + 2),
                              at<double2>(a, X.oB2) + X.cs[s3], X.cols, sa, K, n));
        }
        pr.push_back(Prod{at<double2>(a, X.oXB), K, at<double2>(a, X.oB2), X.cols, at<double2>(a, X.oT), X.cols, X.rows,
                          X.cols, K, OP_N, 1.0, 0});
        check_prod(ck, "B: product", pr.back(), sa, sa, sa);
        wc += 8.0 * (double)X.rows * X.cols * K;
        // scatter theta rows (s1, s2, a) x columns (s3, b) into the compact layout
        for (int s1 = 0; s1 < d; ++s1)
          for (int s2 = 0; s2 < d; ++s2) {
            const int al = X.c - s1 - s2, na = P.rl.count(al);
            if (na == 0) continue;
            for (int s3 = 0; s3 < d; ++s3) {
              const int be = X.c + s3, nb_ = P.rr.count(be);
              if (nb_ == 0) continue;
              const int dl = s1 + s2 + s3, sgi = sg.idx[(s1 * d + s2) * d + s3];
              const long long cbase = P.cb[dl][al - P.rl.lo()];
              const long long off = P.tD[dl] + (long long)sgi * P.NDl[dl] + cbase;
              sc.push_back(scatter(ck, "B: theta", at<double2>(a, P.oTh) + off, nb_,
                                   span_of(a + P.oTh, 16 * (size_t)P.theta_n),
                                   at<double2>(a, X.oT) + (size_t)X.rs[s1 * d + s2] * X.cols + X.cs[s3], X.cols, sa, na,
                                   nb_));
            }
          }
      }
    }
    if (!ck.ok) return TEBD_ERR_STATE;
    ProfScope ps(c, TEBD_PROF_CONTRACT, wc);
    if (int r = launch_moves(c, mv)) return r;
    if (int r = run_prods(c, pr, e_con)) return r;
    if (int r = launch_moves(c, sc)) return r;
  }
  // ---- the gate: C_Delta = G_Delta theta~_Delta (one product per Delta)
  {
    std::vector<Prod> pr;
    double wc = 0.0;
    for (size_t t = 0; t < nt; ++t) {
      Triple& T = ts[t];
      [[maybe_unused]] const int d = T.h->d;
      [[maybe_unused]] const SigmaTable& sg = sgs[d];
      const size_t gsz = (size_t)sgs[T.h->d].gsz;
      tebd_ctx* o = T.h;
      Plan& P = pl[t];
      char* a = T.h->u1w->slots[T.slot].a1.base;
      const double2* Gt = o->Gblk + ((size_t)tidx * (o->L - 2) + T.i) * gsz;
      for (int dl = 0; dl < sg.nDelta; ++dl) {
        const int nd = sg.nD[dl];
        const long long N = P.NDl[dl];
        if (N == 0) continue;
        pr.push_back(Prod{Gt + sg.gbo[dl], nd, at<double2>(a, P.oTh) + P.tD[dl], N, at<double2>(a, P.oC) + P.tD[dl], N,
                          nd, (int)N, nd, OP_N, 1.0, 0});
        check_prod(ck, "gate", pr.back(), span_of(o->Gblk, 16 * o->Gblk_n),
                   span_of(a + P.oTh, 16 * (size_t)P.theta_n), span_of(a + P.oC, 16 * (size_t)P.theta_n));
        wc += 8.0 * (double)nd * nd * N;
      }
    }
    if (!ck.ok) return TEBD_ERR_STATE;
    ProfScope ps(c, TEBD_PROF_CONTRACT, wc);
    if (int r = launch_gate_blocks(c, pr)) return r;
  }
  // ---- the first cut: pack its blocks from the compact C
  {
    std::vector<Move> mv;
    for (size_t t = 0; t < nt; ++t) {
      Triple& T = ts[t];
      [[maybe_unused]] const int d = T.h->d;
      [[maybe_unused]] const SigmaTable& sg = sgs[d];
      tebd_ctx* o = T.h;
      Plan& P = pl[t];
      char* a = T.h->u1w->slots[T.slot].a1.base;
      const Span sa = arena_span(T.h->u1w->slots[T.slot].a1);
      for (CutBlk& B : P.cut1.blk) {
        for (int s1 = 0; s1 < d; ++s1) {
          const int al = B.c - s1, na = P.rl.count(al);
          if (na == 0) continue;
          mv.push_back(gather(ck, "cut 1: lambda", o->lam[T.i] + P.rl.start(al), 1, lam_span(o, T.i),
                              at<double>(a, B.oLam) + B.rs[s1], 1, sa, na, 1, true));
          for (int s2 = 0; s2 < d; ++s2)
            for (int s3 = 0; s3 < d; ++s3) {
              const int be = B.c + s2 + s3, nb_ = P.rr.count(be);
              if (nb_ == 0) continue;
              const int dl = s1 + s2 + s3, sgi = sg.idx[(s1 * d + s2) * d + s3];
              const long long off = P.tD[dl] + (long long)sgi * P.NDl[dl] + P.cb[dl][al - P.rl.lo()];
              mv.push_back(gather(ck, "cut 1: C", at<double2>(a, P.oC) + off, nb_,
                                  span_of(a + P.oC, 16 * (size_t)P.theta_n),
                                  at<double2>(a, B.oP) + (size_t)B.rs[s1] * B.n + B.cs[s2 * d + s3], B.n, sa, na, nb_));
            }
        }
      }
    }
    if (!ck.ok) return TEBD_ERR_STATE;
    ProfScope ps(c, TEBD_PROF_GRAM, 0.0);
    if (int r = launch_moves(c, mv)) return r;
  }
  std::vector<Cut*> cuts(nt);
  std::vector<char*> bases(nt);
  std::vector<double*> lam_out(nt);
  for (size_t t = 0; t < nt; ++t) {
    cuts[t] = &pl[t].cut1;
    bases[t] = ts[t].h->u1w->slots[ts[t].slot].a1.base;
    lam_out[t] = ts[t].h->lam[ts[t].i + 1];
  }
  if (int r = decompose(c, cuts, bases, lam_out)) return r;
  if (int r = kept_vectors(c, cuts, bases)) return r;
  // ---- B_i = P1 W^+ / ||s|| per block, scattered into the dense site tensor
  {
    std::vector<Prod> pr;
    std::vector<Move> sc;
    double wc = 0.0;
    for (size_t t = 0; t < nt; ++t) {
      Triple& T = ts[t];
      [[maybe_unused]] const int d = T.h->d;
      [[maybe_unused]] const SigmaTable& sg = sgs[d];
      tebd_ctx* o = T.h;
      Plan& P = pl[t];
      char* a = T.h->u1w->slots[T.slot].a1.base;
      const Span sa = arena_span(T.h->u1w->slots[T.slot].a1);
      const int chi1 = P.cut1.chi;
      if (cudaMemsetAsync(o->B[T.i], 0, 16 * (size_t)T.chl * d * chi1, s) != cudaSuccess) return fail_cuda(c);
      for (CutBlk& B : P.cut1.blk) {
        if (B.cnt == 0) continue;
        pr.push_back(Prod{at<double2>(a, B.oP), B.n, at<double2>(a, B.oW), B.n, at<double2>(a, B.oOut), B.cnt, B.b,
                          B.cnt, B.n, OP_C, 1.0 / P.cut1.norm, 0});
        check_prod(ck, "rebuild 1", pr.back(), sa, sa, sa);
        wc += 8.0 * (double)B.b * B.cnt * B.n;
        for (int s1 = 0; s1 < d; ++s1) {
          const int al = B.c - s1, na = P.rl.count(al);
          if (na == 0) continue;
          const long long base = ((long long)P.rl.start(al) * d + s1) * chi1 + B.kst;
          sc.push_back(scatter(ck, "rebuild 1: B_i", o->B[T.i] + base, (long long)d * chi1, site_span(o, T.i),
                               at<double2>(a, B.oOut) + (size_t)B.rs[s1] * B.cnt, B.cnt, sa, na, B.cnt));
        }
      }
    }
    if (!ck.ok) return TEBD_ERR_STATE;
    ProfScope ps(c, TEBD_PROF_CONTRACT, wc);
    if (int r = run_prods(c, pr, e_con)) return r;
    if (int r = launch_moves(c, sc)) return r;
  }
  // ---- the second cut: R = diag(s) V1^+ with rows (s2, k) and columns (s3, b)
  for (size_t t = 0; t < nt; ++t) {
    Triple& T = ts[t];
    [[maybe_unused]] const int d = T.h->d;
    [[maybe_unused]] const SigmaTable& sg = sgs[d];
    tebd_ctx* o = T.h;
    Plan& P = pl[t];
    std::vector<int> q1;
    for (const CutBlk& B : P.cut1.blk) q1.insert(q1.end(), B.cnt, B.c);
    P.r1n = runs_of(q1);
    Bump bp;
    P.cut2.chi_cap = std::min(o->chi_max, o->cap[T.i + 2]);
    P.cut2.w_cut = o->w_cut;
    P.cut2.eps_rel = o->eps_rel;
    for (int cq = P.r1n.lo(); cq <= P.r1n.hi() + d - 1; ++cq) {
      CutBlk B{};
      B.c = cq;
      B.rs.assign(d, 0);
      B.cs.assign(d, 0);
      for (int s2 = 0; s2 < d; ++s2) { B.rs[s2] = B.b; B.b += P.r1n.count(cq - s2); }
      for (int s3 = 0; s3 < d; ++s3) { B.cs[s3] = B.n; B.n += P.rr.count(cq + s3); }
      if (B.b == 0 || B.n == 0) continue;
      B.kmax = std::min({B.b, B.n, P.cut2.chi_cap});
      P.cut2.blk.push_back(B);
    }
    layout_cut(P.cut2, bp);
    if (int r = ensure_arena(c, T.h->u1w->slots[T.slot].a2, bp.used)) return r;
  }
  {
    std::vector<Move> mv;
    for (size_t t = 0; t < nt; ++t) {
      Triple& T = ts[t];
      [[maybe_unused]] const int d = T.h->d;
      [[maybe_unused]] const SigmaTable& sg = sgs[d];
      tebd_ctx* o = T.h;
      Plan& P = pl[t];
      char* a1 = T.h->u1w->slots[T.slot].a1.base;
      char* a = T.h->u1w->slots[T.slot].a2.base;
      const Span sa1 = arena_span(T.h->u1w->slots[T.slot].a1), sa = arena_span(T.h->u1w->slots[T.slot].a2);
      for (CutBlk& B : P.cut2.blk) {
        for (int s2 = 0; s2 < d; ++s2) {
          const int c1 = B.c - s2, nk = P.r1n.count(c1);
          if (nk == 0) continue;
          const CutBlk* V = nullptr;  // the first cut's block of charge c1
          for (const CutBlk& X : P.cut1.blk)
            if (X.c == c1) V = &X;
          if (!V) return TEBD_ERR_STATE;
          mv.push_back(gather(ck, "cut 2: lambda", o->lam[T.i + 1] + V->kst, 1, lam_span(o, T.i + 1),
                              at<double>(a, B.oLam) + B.rs[s2], 1, sa, nk, 1, true));
          for (int s3 = 0; s3 < d; ++s3) {
            const int nb_ = P.rr.count(B.c + s3);
            if (nb_ == 0) continue;
            const double2* src = at<double2>(a1, V->oW) + V->cs[s2 * d + s3];
            mv.push_back(gather(ck, "cut 2: V1", src, V->n, sa1, at<double2>(a, B.oP) + (size_t)B.rs[s2] * B.n + B.cs[s3],
                                B.n, sa, nk, nb_));
          }
        }
      }
    }
    if (!ck.ok) return TEBD_ERR_STATE;
    ProfScope ps(c, TEBD_PROF_GRAM, 0.0);
    if (int r = launch_moves(c, mv)) return r;
  }
  for (size_t t = 0; t < nt; ++t) {
    cuts[t] = &pl[t].cut2;
    bases[t] = ts[t].h->u1w->slots[ts[t].slot].a2.base;
    lam_out[t] = ts[t].h->lam[ts[t].i + 2];
  }
  if (int r = decompose(c, cuts, bases, lam_out)) return r;
  if (int r = kept_vectors(c, cuts, bases)) return r;
  // ---- B_{i+2} = V2^+ and B_{i+1} = V1^+ V2 / ||s2||, scattered into the dense site tensors
  {
    std::vector<Prod> pr;
    std::vector<Move> sc;
    double wc = 0.0;
    for (size_t t = 0; t < nt; ++t) {
      Triple& T = ts[t];
      [[maybe_unused]] const int d = T.h->d;
      [[maybe_unused]] const SigmaTable& sg = sgs[d];
      tebd_ctx* o = T.h;
      Plan& P = pl[t];
      char* a = T.h->u1w->slots[T.slot].a2.base;
      const Span sa = arena_span(T.h->u1w->slots[T.slot].a2);
      const int chi1 = P.cut1.chi, chi2 = P.cut2.chi;
      if (cudaMemsetAsync(o->B[T.i + 2], 0, 16 * (size_t)chi2 * d * T.chr, s) != cudaSuccess ||
          cudaMemsetAsync(o->B[T.i + 1], 0, 16 * (size_t)chi1 * d * chi2, s) != cudaSuccess)
        return fail_cuda(c);
      for (CutBlk& B : P.cut2.blk) {
        if (B.cnt == 0) continue;
        for (int s3 = 0; s3 < d; ++s3) {
          const int be = B.c + s3, nb_ = P.rr.count(be);
          if (nb_ == 0) continue;
          const long long base = ((long long)B.kst * d + s3) * T.chr + P.rr.start(be);
          sc.push_back(scatter(ck, "rebuild 2: B_i+2", o->B[T.i + 2] + base, (long long)d * T.chr, site_span(o, T.i + 2),
                               at<double2>(a, B.oW) + B.cs[s3], B.n, sa, B.cnt, nb_));
        }
        pr.push_back(Prod{at<double2>(a, B.oP), B.n, at<double2>(a, B.oW), B.n, at<double2>(a, B.oOut), B.cnt, B.b,
                          B.cnt, B.n, OP_C, 1.0 / P.cut2.norm, 0});
        check_prod(ck, "rebuild 2", pr.back(), sa, sa, sa);
        wc += 8.0 * (double)B.b * B.cnt * B.n;
        for (int s2 = 0; s2 < d; ++s2) {
          const int c1 = B.c - s2, nk = P.r1n.count(c1);
          if (nk == 0) continue;
          const long long base = ((long long)P.r1n.start(c1) * d + s2) * chi2 + B.kst;
          sc.push_back(scatter(ck, "rebuild 2: B_i+1", o->B[T.i + 1] + base, (long long)d * chi2, site_span(o, T.i + 1),
                               at<double2>(a, B.oOut) + (size_t)B.rs[s2] * B.cnt, B.cnt, sa, nk, B.cnt));
        }
      }
    }
    if (!ck.ok) return TEBD_ERR_STATE;
    ProfScope ps(c, TEBD_PROF_CONTRACT, wc);
    if (int r = run_prods(c, pr, e_con)) return r;
    if (int r = launch_moves(c, sc)) return r;
  }
  for (size_t t = 0; t < nt; ++t) {
    Triple& T = ts[t];
    [[maybe_unused]] const int d = T.h->d;
    [[maybe_unused]] const SigmaTable& sg = sgs[d];
    tebd_ctx* o = T.h;
    Plan& P = pl[t];
    std::vector<int> q1, q2;
    for (const CutBlk& B : P.cut1.blk) q1.insert(q1.end(), B.cnt, B.c);
    for (const CutBlk& B : P.cut2.blk) q2.insert(q2.end(), B.cnt, B.c);
    o->q[T.i + 1] = q1;
    o->q[T.i + 2] = q2;
    o->chi[T.i + 1] = P.cut1.chi;
    o->chi[T.i + 2] = P.cut2.chi;
    o->w_total += P.cut1.w + P.cut2.w;
    o->gate_updates += 1;
  }
  return TEBD_OK;
}

}  // namespace

int update_chunk_u1(tebd_ctx* c, std::vector<Triple>& ts, int tidx) {
  if (!c->u1w) return TEBD_ERR_STATE;
  for (const Triple& T : ts)
    if (!T.h->u1w || (int)T.h->u1w->slots.size() <= T.slot) return TEBD_ERR_STATE;
  if (int r = stage_begin_chunk(c)) return r;
  const int r = update_chunk_u1_body(c, ts, tidx);
  // the staging buffer of this chunk is reusable once the work issued so far has run
  const int re = stage_end_chunk(c);
  return r != TEBD_OK ? r : re;
}

namespace {

// ---- randomized range finder for the dense form (the cheaper SVD of Sec. V) -------------

__global__ void k_fill(double* __restrict__ x, size_t n, double v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) x[i] = v;
}

// out[t] = ||M_t||_F^2 with M_t[r][:] = lam_t[r / d] X_t[r][:] (m_t x n_t, row-major)
struct FrobArgs {
  const double2* X;
  const double* lam;
  int m, n, d;
  double* out;
};
__global__ void k_frob(const FrobArgs* __restrict__ fa) {
  const FrobArgs F = fa[blockIdx.x];
  __shared__ double sh[32];
  double acc = 0.0;
  for (long long e = threadIdx.x; e < (long long)F.m * F.n; e += blockDim.x) {
    const int r = (int)(e / F.n);
    const double l = F.lam[r / F.d];
    const double2 v = F.X[e];
    acc = fma(l * l, fma(v.x, v.x, v.y * v.y), acc);
  }
  acc = warp_sum_d(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    *F.out = t;
  }
}

// One cut of one block for a row matrix P (rows x cols) already in the arena's layout:
// every direction kept (an orthonormal basis of the row space), or rule T (final).
void one_block_cut(Cut& cut, int rows, int cols, int chi_cap, double w_cut, double eps_rel, Bump& bp) {
  cut = Cut{};
  CutBlk B{};
  B.b = rows;
  B.n = cols;
  B.kmax = std::min({rows, cols, chi_cap});
  cut.blk.push_back(B);
  cut.chi_cap = chi_cap;
  cut.w_cut = w_cut;
  cut.eps_rel = eps_rel;
  layout_cut(cut, bp);
}

// The row matrix of a triple's cut: M[r][:] = lam[r / d] X[r][:], m x n (dense form).
struct RandIn {
  const double2* X;
  const double* lam;
  int m, n, d;
};

// Products with M on the engine of the path: C (rows x N) = A op(M) with op(M) = M (then
// the reduction runs over the rows of M, scaled by lam) or M^+ (then the columns of the
// result are the rows of M, scaled by lam); A is rows x K (or Omega^+ when omega).
void prod_with_M(tebd_ctx* c, Gemm& gN, Gemm& gC, std::vector<OzProb>& oz, const RandIn& in, const double2* A,
                 int rows, bool adjoint, bool omega, double2* C) {
  const bool mixed = c->precision >= 1;
  if (!adjoint) {  // C = A M: A rows x m, C rows x n
    if (mixed) {
      OzProb q{};
      q.a = OzOperand{A, in.m, 1, in.lam, in.d, 0};
      q.b = OzOperand{in.X, 1, in.n, nullptr, 1, 0};
      q.M = rows; q.N = in.n; q.K = in.m; q.C = C; q.ldc = in.n; q.alpha = 1.0; q.row_div = q.col_div = 1;
      oz.push_back(q);
    } else {
      GemmProb& p = gN.add(rows, in.n, in.m, A, in.m, in.X, in.n, C, in.n);
      p.s_red = in.lam;
      p.red_div = in.d;
    }
  } else {  // C = A M^+: A rows x n (or Omega^+ with Omega n x rows), C rows x m
    if (mixed) {
      OzProb q{};
      q.a = omega ? OzOperand{A, 1, rows, nullptr, 1, 1} : OzOperand{A, in.n, 1, nullptr, 1, 0};
      q.b = OzOperand{in.X, in.n, 1, nullptr, 1, 1};
      q.M = rows; q.N = in.m; q.K = in.n; q.C = C; q.ldc = in.m; q.alpha = 1.0;
      q.s_col = in.lam; q.row_div = 1; q.col_div = in.d;
      oz.push_back(q);
    } else {  // omega: gC computes Omega^+ M^+ (both operands conjugate-transposed); else gN is (N, C)
      GemmProb& p = (omega ? gC : gN).add(rows, in.m, in.n, A, omega ? rows : in.n, in.X, in.n, C, in.m);
      p.s_col = in.lam;
      p.col_div = in.d;
    }
  }
}

int run_M_prods(tebd_ctx* c, Gemm& gN, Gemm& gC, std::vector<OzProb>& oz, double w) {
  ProfScope ps(c, TEBD_PROF_PROJECT, w);
  if (c->precision >= 1) {
    size_t need = 0;
    for (const OzProb& q : oz) need = std::max(need, oz_workspace_bytes(q.M, q.N, q.K, false));
    if (int r = ensure_ring(c, need)) return r;
    for (size_t j = 0; j < oz.size(); ++j) oz[j].ws = c->u1w->ring[j % OZ_MAXP];
    c->launches += oz_gemm_launch(oz, c->d_status, c->stream);
  } else {
    c->launches += gN.launch(c->stream);
    c->launches += gC.launch(c->stream);
  }
  return check_launch(c);
}

}  // namespace

namespace {

int rand_cut_body(tebd_ctx* c, std::vector<Triple>& ts, bool second) {
  const size_t nt = ts.size();
  std::vector<RandIn> in(nt);
  std::vector<int> ell(nt);
  std::vector<U1Slot*> sl(nt);
  for (size_t t = 0; t < nt; ++t) {
    Triple& T = ts[t];
    tebd_ctx* o = T.h;
    const Slot& S = o->slots[T.slot];
    if (!o->omega_fn) return TEBD_ERR_STATE;
    in[t] = second ? RandIn{S.V1h, o->lam[T.i + 1], T.m2, T.n2, o->d} : RandIn{S.Cb, o->lam[T.i], T.m1, T.n1, o->d};
    ell[t] = std::min({o->chi_max + o->oversample, in[t].m, in[t].n});
    sl[t] = &o->u1w->slots[T.slot];
  }
  // Omega of each decomposition from the caller (an input, never drawn here) into arena a2,
  // and ||M||_F^2 beside it
  std::vector<FrobArgs> fa(nt);
  std::vector<double> host;
  for (size_t t = 0; t < nt; ++t) {
    const size_t ob = align256(16 * (size_t)in[t].n * ell[t]);
    if (int r = ensure_arena(c, sl[t]->a2, ob + 256)) return r;
  }
  for (size_t t = 0; t < nt; ++t) {
    Triple& T = ts[t];
    host.assign(2 * (size_t)in[t].n * ell[t], 0.0);
    T.h->omega_fn(T.call + (second ? 1 : 0), in[t].n, ell[t], host.data(), T.h->omega_ctx);
    for (double x : host)
      if (!is_fin(x)) return TEBD_ERR_ARG;
    // a pageable copy is staged before the call returns, so host can be refilled at once
    if (cudaMemcpy(sl[t]->a2.base, host.data(), 8 * host.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail_cuda(c);
    fa[t] = FrobArgs{in[t].X, in[t].lam, in[t].m, in[t].n, in[t].d,
                     reinterpret_cast<double*>(sl[t]->a2.base + align256(16 * (size_t)in[t].n * ell[t]))};
  }
  {
    int err = TEBD_OK;
    FrobArgs* dfa = stage(c, fa, &err);
    if (err) return err;
    k_frob<<<(unsigned)nt, 256, 0, c->stream>>>(dfa);
    c->launches += 1;
    if (int r = check_launch(c)) return r;
  }
  if (int r = ensure_back(c, nt + 2)) return r;
  for (size_t t = 0; t < nt; ++t) cudaMemcpyAsync(c->u1w->h_back + t, fa[t].out, 8, cudaMemcpyDeviceToHost, c->stream);
  if (int r = sync(c)) return r;
  std::vector<double> frob(nt);
  for (size_t t = 0; t < nt; ++t) {
    frob[t] = c->u1w->h_back[t];
    if (!is_fin(frob[t]) || !(frob[t] > 0.0)) {
      c->sticky = TEBD_ERR_NONFINITE;
      return TEBD_ERR_NONFINITE;
    }
  }
  // Yh = Omega^+ M^+ (l x m); q times Zh = Q M (r x n), Yh = Z M^+ (r x m); C = Q M (r x n).
  // Every intermediate row matrix is replaced by an orthonormal basis of its row space (a
  // one-block cut that keeps every direction above the Gram floor); the last, C, is cut by
  // rule T with the tail from ||M||_F^2.  The steps alternate between the slot's arenas.
  const int nsteps = 2 + 2 * std::max(0, c->power_iters);
  std::vector<Cut> prev(nt), cur(nt);
  std::vector<int> rows(ell);
  std::vector<char*> pbase(nt);
  for (int stp = 0; stp < nsteps; ++stp) {
    const bool final_step = (stp == nsteps - 1);
    const bool adj = (stp % 2 == 0);  // the Yh steps multiply by M^+
    std::vector<Cut*> cp(nt);
    std::vector<char*> bases(nt);
    std::vector<double*> lo(nt);
    std::vector<size_t> lam_off(nt);
    for (size_t t = 0; t < nt; ++t) {
      Triple& T = ts[t];
      tebd_ctx* o = T.h;
      const int cols = adj ? in[t].m : in[t].n;
      Bump bp;
      if (final_step)
        one_block_cut(cur[t], rows[t], cols, std::min(o->chi_max, o->cap[T.i + (second ? 2 : 1)]), o->w_cut,
                      o->eps_rel, bp);
      else
        one_block_cut(cur[t], rows[t], cols, std::min(rows[t], cols), 0.0, 0.0, bp);
      cur[t].total_fixed = final_step ? frob[t] : -1.0;
      lam_off[t] = bp.take(8 * (size_t)rows[t]);
      U1Arena& dst = (stp % 2 == 0) ? sl[t]->a1 : sl[t]->a2;
      if (int r = ensure_arena(c, dst, bp.used)) return r;
      bases[t] = dst.base;
      cp[t] = &cur[t];
      lo[t] = final_step ? o->lam[T.i + (second ? 2 : 1)] : at<double>(dst.base, lam_off[t]);
    }
    // the row matrix of this step from the previous basis (or Omega)
    {
      Gemm gN(true, OP_N, OP_N), gC(true, OP_C, OP_C), gNC(true, OP_N, OP_C);
      std::vector<OzProb> oz;
      double w = 0.0;
      for (size_t t = 0; t < nt; ++t) {
        const CutBlk& B = cur[t].blk[0];
        double2* P = at<double2>(bases[t], B.oP);
        if (stp == 0) {
          prod_with_M(c, gN, gC, oz, in[t], reinterpret_cast<const double2*>(sl[t]->a2.base), rows[t], true, true, P);
        } else {
          const CutBlk& Bp = prev[t].blk[0];
          const double2* Wp = at<double2>(pbase[t], Bp.oW);
          prod_with_M(c, adj ? gNC : gN, gC, oz, in[t], Wp, rows[t], adj, false, P);
        }
        w += 8.0 * (double)rows[t] * in[t].m * in[t].n;
        k_fill<<<(rows[t] + 255) / 256, 256, 0, c->stream>>>(at<double>(bases[t], B.oLam), (size_t)rows[t], 1.0);
        c->launches += 1;
      }
      if (int r = run_M_prods(c, gN, gC, oz, w)) return r;
      c->launches += gNC.launch(c->stream);
      if (int r = check_launch(c)) return r;
    }
    if (int r = decompose(c, cp, bases, lo)) return r;
    if (int r = kept_vectors(c, cp, bases)) return r;
    for (size_t t = 0; t < nt; ++t) {
      rows[t] = cur[t].chi;
      pbase[t] = bases[t];
    }
    std::swap(prev, cur);
  }
  // the kept right vectors into the site workspace (cut 1: V1^+) or tensor (cut 2: B_{i+2})
  for (size_t t = 0; t < nt; ++t) {
    Triple& T = ts[t];
    tebd_ctx* o = T.h;
    const Cut& F = prev[t];
    const CutBlk& B = F.blk[0];
    double2* dst = second ? o->B[T.i + 2] : o->slots[T.slot].V1h;
    if (cudaMemcpyAsync(dst, at<double2>(pbase[t], B.oW), 16 * (size_t)F.chi * B.n, cudaMemcpyDeviceToDevice,
                        c->stream) != cudaSuccess)
      return fail_cuda(c);
    if (second) { T.chi2 = F.chi; T.norm2 = F.norm; T.w2 = F.w; }
    else { T.chi1 = F.chi; T.norm1 = F.norm; T.w1 = F.w; }
  }
  return check_launch(c);
}

}  // namespace

int rand_cut(tebd_ctx* c, std::vector<Triple>& ts, bool second) {
  if (!c->u1w) return TEBD_ERR_STATE;
  for (const Triple& T : ts)
    if (!T.h->u1w || (int)T.h->u1w->slots.size() <= T.slot) return TEBD_ERR_STATE;
  if (int r = stage_begin_chunk(c)) return r;
  const int r = rand_cut_body(c, ts, second);
  const int re = stage_end_chunk(c);
  return r != TEBD_OK ? r : re;
}

namespace {

// Nearest-neighbour correlators C_k = <b+_k b_{k+1}> of every bond from the charge blocks of
// the canonical form (eq. (5)): with c, c' indices of the middle bond,
//   C = sum_{c, c'} X[c, c'] Y[c', c],
//   X[c, c'] = sum_{a, s} lam_a^2 sqrt(s+1) conj(B_k[a, s+1, c]) B_k[a, s, c'],
//   Y[c', c] = sum_{t, b} sqrt(t+1) B_{k+1}[c', t+1, b] conj(B_{k+1}[c, t, b]),
// and X, Y vanish unless q(c) = q(c') + 1: for each charge v of c' one product pair
// over the rows (a, s) with q(a) + s = v and the columns (t, b) with q(b) = v + 1 + t.
int correlators_body(tebd_ctx* h, double2* out) {
  const int L = h->L, d = h->d;
  Checker ck;
  struct VB { int k, v, Kx, Ky, nu, nv; size_t oP, oB, oQ, oU, oX, oY, oLam, oF, oW; std::vector<int> rx, cy; };
  std::vector<VB> vb;
  Bump bp;
  for (int k = 0; k + 1 < L; ++k) {
    const Runs rl = runs_of(h->q[k]), rm = runs_of(h->q[k + 1]), rr = runs_of(h->q[k + 2]);
    for (int v = rm.lo(); v <= rm.hi(); ++v) {
      const int nv = rm.count(v), nu = rm.count(v + 1);
      if (nv == 0 || nu == 0) continue;
      VB X{};
      X.k = k; X.v = v; X.nu = nu; X.nv = nv;
      X.rx.assign(d, 0);
      X.cy.assign(d, 0);
      for (int s1 = 0; s1 + 1 < d; ++s1) { X.rx[s1] = X.Kx; X.Kx += rl.count(v - s1); }
      for (int t = 0; t + 1 < d; ++t) { X.cy[t] = X.Ky; X.Ky += rr.count(v + 1 + t); }
      if (X.Kx == 0 || X.Ky == 0) continue;
      X.oP = bp.take(16 * (size_t)X.Kx * nu);
      X.oB = bp.take(16 * (size_t)X.Kx * nv);
      X.oQ = bp.take(16 * (size_t)nv * X.Ky);
      X.oU = bp.take(16 * (size_t)nu * X.Ky);
      X.oX = bp.take(16 * (size_t)nu * nv);
      X.oY = bp.take(16 * (size_t)nv * nu);
      X.oLam = bp.take(8 * (size_t)X.Kx);
      X.oF = bp.take(8 * (size_t)X.Kx);
      X.oW = bp.take(8 * (size_t)(X.Kx + X.Ky));
      vb.push_back(X);
    }
  }
  if (cudaMemsetAsync(out, 0, sizeof(double2) * (L - 1), h->stream) != cudaSuccess) return fail_cuda(h);
  if (vb.empty()) return TEBD_OK;
  if (int r = ensure_arena(h, h->u1w->meas, bp.used)) return r;
  char* a = h->u1w->meas.base;
  const Span sa = arena_span(h->u1w->meas);
  std::vector<Move> mv;
  std::vector<double> wts;  // sqrt(s+1) per row of X's reduction, then sqrt(t+1) per column of Y's
  std::vector<size_t> woff;
  for (VB& X : vb) {
    const int k = X.k, v = X.v, chl = h->chi[k], chm = h->chi[k + 1], chr = h->chi[k + 2];
    const Runs rl = runs_of(h->q[k]), rm = runs_of(h->q[k + 1]), rr = runs_of(h->q[k + 2]);
    woff.push_back(wts.size());
    for (int s1 = 0; s1 + 1 < d; ++s1) {
      const int na = rl.count(v - s1);
      if (na == 0) continue;
      const long long a0 = rl.start(v - s1);
      mv.push_back(gather(ck, "measure: B_k shifted", h->B[k] + (a0 * d + s1 + 1) * chm + rm.start(v + 1),
                          (long long)d * chm, site_span(h, k), at<double2>(a, X.oP) + (size_t)X.rx[s1] * X.nu, X.nu, sa,
                          na, X.nu));
      mv.push_back(gather(ck, "measure: B_k", h->B[k] + (a0 * d + s1) * chm + rm.start(v), (long long)d * chm,
                          site_span(h, k), at<double2>(a, X.oB) + (size_t)X.rx[s1] * X.nv, X.nv, sa, na, X.nv));
      mv.push_back(gather(ck, "measure: lambda", h->lam[k] + a0, 1, lam_span(h, k), at<double>(a, X.oLam) + X.rx[s1],
                          1, sa, na, 1, true));
      wts.insert(wts.end(), na, std::sqrt((double)(s1 + 1)));
    }
    for (int t = 0; t + 1 < d; ++t) {
      const int nb_ = rr.count(v + 1 + t);
      if (nb_ == 0) continue;
      const long long b0 = rr.start(v + 1 + t);
      mv.push_back(gather(ck, "measure: B_k+1 shifted", h->B[k + 1] + ((long long)rm.start(v) * d + t + 1) * chr + b0,
                          (long long)d * chr, site_span(h, k + 1), at<double2>(a, X.oQ) + X.cy[t], X.Ky, sa, X.nv, nb_));
      mv.push_back(gather(ck, "measure: B_k+1", h->B[k + 1] + ((long long)rm.start(v + 1) * d + t) * chr + b0,
                          (long long)d * chr, site_span(h, k + 1), at<double2>(a, X.oU) + X.cy[t], X.Ky, sa, X.nu, nb_));
      wts.insert(wts.end(), nb_, std::sqrt((double)(t + 1)));
    }
    (void)chl;
  }
  if (!ck.ok) return TEBD_ERR_STATE;
  if (int r = launch_moves(h, mv)) return r;
  int err = TEBD_OK;
  double* dw = stage(h, wts, &err);
  if (err) return err;
  // the two products per block: on the FP64 CUDA cores, or (precision 1 and 2) on the
  // exact-digit engine, whose results carry FP64 accuracy
  const bool tc = h->precision >= 1;
  Gemm gx(true, OP_C, OP_N), gy(true, OP_N, OP_C);
  std::vector<OzProb> oz;
  size_t need = 0;
  std::vector<TraceBlk> tb;
  std::vector<TraceBond> bonds;
  for (size_t i = 0; i < vb.size(); ++i) {
    VB& X = vb[i];
    const double* w = dw + woff[i];
    if (cudaMemcpyAsync(a + X.oW, w, 8 * (size_t)(X.Kx + X.Ky), cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
      return fail_cuda(h);
    k_lam2w<<<(X.Kx + 255) / 256, 256, 0, h->stream>>>(at<double>(a, X.oLam), at<double>(a, X.oW), at<double>(a, X.oF),
                                                       X.Kx);
    h->launches += 1;
    if (tc) {  // X = P^+ diag(f) B (nu x nv over Kx), Y = Q diag(w) U^+ (nv x nu over Ky)
      OzProb qx{};
      qx.a = OzOperand{at<double2>(a, X.oP), 1, X.nu, at<double>(a, X.oF), 1, 1};
      qx.b = OzOperand{at<double2>(a, X.oB), 1, X.nv, nullptr, 1, 0};
      qx.M = X.nu; qx.N = X.nv; qx.K = X.Kx; qx.C = at<double2>(a, X.oX); qx.ldc = X.nv; qx.alpha = 1.0;
      qx.row_div = qx.col_div = 1;
      OzProb qy{};
      qy.a = OzOperand{at<double2>(a, X.oQ), X.Ky, 1, at<double>(a, X.oW) + X.Kx, 1, 0};
      qy.b = OzOperand{at<double2>(a, X.oU), X.Ky, 1, nullptr, 1, 1};
      qy.M = X.nv; qy.N = X.nu; qy.K = X.Ky; qy.C = at<double2>(a, X.oY); qy.ldc = X.nu; qy.alpha = 1.0;
      qy.row_div = qy.col_div = 1;
      need = std::max({need, oz_workspace_bytes(qx.M, qx.N, qx.K, false), oz_workspace_bytes(qy.M, qy.N, qy.K, false)});
      oz.push_back(qx);
      oz.push_back(qy);
    } else {
      GemmProb& px = gx.add(X.nu, X.nv, X.Kx, at<double2>(a, X.oP), X.nu, at<double2>(a, X.oB), X.nv,
                            at<double2>(a, X.oX), X.nv);
      px.s_red = at<double>(a, X.oF);
      GemmProb& py = gy.add(X.nv, X.nu, X.Ky, at<double2>(a, X.oQ), X.Ky, at<double2>(a, X.oU), X.Ky,
                            at<double2>(a, X.oY), X.nu);
      py.s_red = at<double>(a, X.oW) + X.Kx;
    }
    if (bonds.empty() || bonds.back().out != out + X.k) bonds.push_back(TraceBond{(int)tb.size(), (int)tb.size(), out + X.k});
    tb.push_back(TraceBlk{at<double2>(a, X.oX), at<double2>(a, X.oY), X.nu, X.nv});
    bonds.back().b1 = (int)tb.size();
  }
  if (tc) {
    if (int r = ensure_ring(h, need)) return r;
    for (size_t j = 0; j < oz.size(); ++j) oz[j].ws = h->u1w->ring[j % OZ_MAXP];
    h->launches += oz_gemm_launch(oz, h->d_status, h->stream);
  } else {
    h->launches += gx.launch(h->stream);
    h->launches += gy.launch(h->stream);
  }
  TraceBlk* dtb = stage(h, tb, &err);
  if (err) return err;
  TraceBond* dbd = stage(h, bonds, &err);
  if (err) return err;
  k_trace_bonds<<<(unsigned)bonds.size(), 256, 0, h->stream>>>(dbd, dtb);
  h->launches += 1;
  return check_launch(h);
}

}  // namespace

int u1_correlators(tebd_ctx* h, double2* out) {
  if (!h->u1w) return TEBD_ERR_STATE;
  if (int r = stage_begin_chunk(h)) return r;
  const int r = correlators_body(h, out);
  const int re = stage_end_chunk(h);
  return r != TEBD_OK ? r : re;
}

int u1_build_gate_blocks(tebd_ctx* c, const std::vector<std::complex<double>>& Gall, size_t ngates) {
  const int d = c->d, D = c->D;
  const SigmaTable sg(d);
  std::vector<std::complex<double>> blk(ngates * (size_t)sg.gsz);
  std::vector<std::vector<int>> members(sg.nDelta);
  for (int x = 0; x < D; ++x) members[x / (d * d) + (x / d) % d + x % d].push_back(x);
  for (size_t g = 0; g < ngates; ++g) {
    const std::complex<double>* G = Gall.data() + g * (size_t)D * D;
    std::complex<double>* out = blk.data() + g * (size_t)sg.gsz;
    for (int dl = 0; dl < sg.nDelta; ++dl) {
      const auto& mem = members[dl];
      const int n = (int)mem.size();
      for (int r = 0; r < n; ++r)
        for (int q = 0; q < n; ++q) out[sg.gbo[dl] + r * n + q] = G[(size_t)mem[r] * D + mem[q]];
    }
  }
  double2* dst = nullptr;
  if (cudaMalloc(&dst, blk.size() * sizeof(double2)) != cudaSuccess) {
    cudaGetLastError();
    return TEBD_ERR_OOM;
  }
  if (cudaMemcpy(dst, blk.data(), blk.size() * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(dst);
    return TEBD_ERR_CUDA;
  }
  if (c->Gblk) cudaFree(c->Gblk);
  c->Gblk = dst;
  c->Gblk_n = blk.size();
  return TEBD_OK;
}

size_t u1_workspace_bytes(const tebd_ctx* c) {
  if (!c->u1w) return 0;
  size_t b = c->u1w->ring_bytes * c->u1w->ring.size() + c->u1w->ering_bytes * c->u1w->ering.size() +
             c->u1w->stage_cap[0] + c->u1w->stage_cap[1];
  for (const U1Slot& s : c->u1w->slots) b += s.a1.cap + s.a2.cap;
  b += c->u1w->meas.cap;
  return b;
}

void u1_release(tebd_ctx* c) {
  if (!c->u1w) return;
  U1Work& w = *c->u1w;
  for (U1Slot& s : w.slots) {
    if (s.a1.base) cudaFree(s.a1.base);
    if (s.a2.base) cudaFree(s.a2.base);
  }
  for (void* p : w.ring) cudaFree(p);
  for (void* p : w.ering) cudaFree(p);
  if (w.meas.base) cudaFree(w.meas.base);
  for (int p = 0; p < 2; ++p) {
    for (auto& b : w.retired[p]) {
      cudaFreeHost(b.first);
      cudaFree(b.second);
    }
    if (w.h_stage[p]) cudaFreeHost(w.h_stage[p]);
    if (w.d_stage[p]) cudaFree(w.d_stage[p]);
    if (w.ev[p]) cudaEventDestroy(w.ev[p]);
  }
  if (w.h_back) cudaFreeHost(w.h_back);
  if (w.d_counts) cudaFree(w.d_counts);
  delete c->u1w;
  c->u1w = nullptr;
}

int u1_alloc_slots(tebd_ctx* c, int nslots) {
  try {
    if (!c->u1w) c->u1w = new U1Work();
  } catch (...) {
    return TEBD_ERR_OOM;
  }
  if ((int)c->u1w->slots.size() < nslots) c->u1w->slots.resize(nslots);
  return TEBD_OK;
}

}  // namespace ptebd
