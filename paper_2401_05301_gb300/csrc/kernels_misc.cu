// Truncation, gathers, state initialisation and observable kernels.
#include "ptebd_internal.h"

#include <algorithm>
#include <cfloat>
#include <cmath>

namespace ptebd {

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return __shfl_sync(0xffffffffu, v, 0);
}

__device__ double block_sum(double v, double* sh) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = (l < nw) ? sh[l] : 0.0;
    t = warp_sum(t);
    if (l == 0) sh[32] = t;
  }
  __syncthreads();
  return sh[32];
}

// ---- truncation (reading of the tolerances of Sec. II B) -----------------------------
// s_k = ||Y_k|| (Y_k = u_k^+ theta'), sorted descending (ties: lower index first);
// p_k = s_k^2 / trace; chi_w = smallest k with sum_{i>k} p_i <= w_cut;
// chi_eps = #{p_k > eps_rel}; chi' = max(1, min(chi_max, chi_w, chi_eps, K)).
// The tail beyond the K computed values is trace - sum_{i<K} s_i^2.
__global__ void k_truncate(const __grid_constant__ TruncBatch tb) {
  const TruncArgs& A = tb.a[blockIdx.x];
  extern __shared__ unsigned char smem_raw[];
  const int K = A.K, n = A.n;
  int P = 1;
  while (P < K) P <<= 1;
  double* s = reinterpret_cast<double*>(smem_raw);
  int* idx = reinterpret_cast<int*>(s + P);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int r = warp; r < K; r += nw) {
    const double2* y = A.Y + (size_t)r * n;
    double acc = 0.0;
    for (int c = lane; c < n; c += 32) acc = fma(y[c].x, y[c].x, fma(y[c].y, y[c].y, acc));
    acc = warp_sum(acc);
    if (lane == 0) { s[r] = sqrt(acc); idx[r] = r; }
  }
  for (int r = K + threadIdx.x; r < P; r += blockDim.x) { s[r] = -1.0; idx[r] = 0x7fffffff; }
  __syncthreads();
  // bitonic sort, descending by s, ascending by idx on ties
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int jx = i ^ stride;
        if (jx > i) {
          const bool desc = ((i & size) == 0);
          const double si = s[i], sj = s[jx];
          const int ii = idx[i], ij = idx[jx];
          // "i before jx" in descending order if si > sj or (si == sj and ii < ij)
          const bool i_first = (si > sj) || (si == sj && ii < ij);
          if (desc != i_first) { s[i] = sj; s[jx] = si; idx[i] = ij; idx[jx] = ii; }
        }
      }
      __syncthreads();
    }
  }
  __shared__ int chi_sh;
  __shared__ double norm_sh;
  if (threadIdx.x == 0) {
    const double total = *A.trace;
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
      double tail = tailK;  // tail(k) = sum_{i >= k} s_i^2 + tailK
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
      atomicExch(A.status, -7);
    }
    chi_sh = chi;
    norm_sh = sqrt(kept);
    *A.chi_out = chi;
    *A.norm_out = norm_sh;
    *A.w_out = w;
  }
  __syncthreads();
  const int chi = chi_sh;
  const double inv = (norm_sh > 0.0) ? 1.0 / norm_sh : 0.0;
  for (int i = threadIdx.x; i < K; i += blockDim.x) {
    A.s_sorted[i] = s[i];
    A.perm[i] = idx[i];
    if (i < chi) A.lam_out[i] = s[i] * inv;
  }
}

struct GatherBatch {
  GatherArgs a[TRUNC_MAXP];
  int n;
};

__global__ void k_gather(const __grid_constant__ GatherBatch gb) {
  const GatherArgs& A = gb.a[blockIdx.y];
  const int k = blockIdx.x;
  if (k >= A.chi) return;
  const double2* src = A.Y + (size_t)A.perm[k] * A.n;
  double2* dst = A.out + (size_t)k * A.n;
  const double s = A.s_sorted[k];
  const double inv = (s > 0.0) ? 1.0 / s : 0.0;
  for (int c = threadIdx.x; c < A.n; c += blockDim.x) {
    const double2 v = src[c];
    dst[c] = make_double2(v.x * inv, v.y * inv);
  }
}

__global__ void k_init_product(double2* const* B, double* const* lam, const int* occ, int L, int d) {
  const int k = blockIdx.x;
  if (threadIdx.x < d) B[k][threadIdx.x] = make_double2(threadIdx.x == occ[k] ? 1.0 : 0.0, 0.0);
  if (threadIdx.x == 0) lam[k][0] = 1.0;
  if (threadIdx.x == 0 && k == L - 1) lam[L][0] = 1.0;
}

struct DensityBatch {
  DensityArgs a[32];
  int n;
};

// n_j = sum_{a,s,b} lam_a^2 |B[a,s,b]|^2 s  (eq. (8) in canonical form)
__global__ void k_densities(const __grid_constant__ DensityBatch db) {
  const DensityArgs& A = db.a[blockIdx.x];
  __shared__ double sh[33];
  const long long total = (long long)A.chl * A.d * A.chr;
  double acc = 0.0;
  for (long long e = threadIdx.x; e < total; e += blockDim.x) {
    const int a = (int)(e / ((long long)A.d * A.chr));
    const int s = (int)((e / A.chr) % A.d);
    const double2 v = A.B[e];
    const double l = A.lam[a];
    const int w = (A.wmode == 1) ? s / A.wd : (A.wmode == 2 ? s % A.wd : s);
    acc += l * l * (double)w * (v.x * v.x + v.y * v.y);
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) *A.out = acc;
}

__global__ void k_shift_left(const double2* B, const double* lam, double2* out, int chl, int d, int chr) {
  const long long total = (long long)chl * d * chr;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(e / ((long long)d * chr));
    const int s = (int)((e / chr) % d);
    const int c = (int)(e % chr);
    double2 v = make_double2(0.0, 0.0);
    if (s < d - 1) {
      const double w = lam[a] * lam[a] * sqrt((double)(s + 1));
      const double2 x = B[((long long)a * d + s + 1) * chr + c];
      v = make_double2(w * x.x, w * x.y);
    }
    out[e] = v;
  }
}

__global__ void k_shift_right(const double2* B, double2* out, int chl, int d, int chr) {
  const long long total = (long long)chl * d * chr;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e / ((long long)d * chr));
    const int t = (int)((e / chr) % d);
    const int b = (int)(e % chr);
    double2 v = make_double2(0.0, 0.0);
    if (t < d - 1) {
      const double w = sqrt((double)(t + 1));
      const double2 x = B[((long long)c * d + t + 1) * chr + b];
      v = make_double2(w * x.x, w * x.y);
    }
    out[e] = v;
  }
}

__global__ void k_trace_product(const double2* X, const double2* Yt, int chi, double2* out) {
  __shared__ double sh[33];
  double re = 0.0, im = 0.0;
  const long long total = (long long)chi * chi;
  for (long long e = threadIdx.x; e < total; e += blockDim.x) {
    const int c = (int)(e / chi), cp = (int)(e % chi);
    const double2 x = X[e], y = Yt[(long long)cp * chi + c];
    re += x.x * y.x - x.y * y.y;
    im += x.x * y.y + x.y * y.x;
  }
  re = block_sum(re, sh);
  im = block_sum(im, sh);
  if (threadIdx.x == 0) *out = make_double2(re, im);
}

__global__ void k_check_finite(const double* x, int n, int* status) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (!isfinite(x[i])) atomicExch(status, -7);
}

int grid_for(long long n) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 4 * 152)); }

}  // namespace

static_assert(sizeof(TruncBatch) < 4000, "kernel parameter block too large");
static_assert(sizeof(GatherBatch) < 4000, "kernel parameter block too large");
static_assert(sizeof(DensityBatch) < 4000, "kernel parameter block too large");

int launch_truncate(const TruncBatch& b, cudaStream_t s) {
  if (b.n == 0) return 0;
  int Kmax = 1;
  for (int i = 0; i < b.n; ++i) Kmax = std::max(Kmax, b.a[i].K);
  int P = 1;
  while (P < Kmax) P <<= 1;
  const size_t smem = (size_t)P * (sizeof(double) + sizeof(int));
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_truncate, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  k_truncate<<<b.n, 512, smem, s>>>(b);
  return 1;
}

namespace {
struct PolarBatch {
  PolarArgs a[TRUNC_MAXP];
  int n;
};
__global__ void k_polar_form(const __grid_constant__ PolarBatch pb) {
  const PolarArgs& a = pb.a[blockIdx.y];
  const int nn = a.n * a.n;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nn; idx += gridDim.x * blockDim.x) {
    const double2 g = a.G[idx];
    a.G[idx] = make_double2((idx / a.n == idx % a.n ? 1.5 : 0.0) - 0.5 * g.x, -0.5 * g.y);
  }
}
}  // namespace

int launch_polar_form(const PolarArgs* a, int n, cudaStream_t s) {
  int launches = 0;
  for (int i0 = 0; i0 < n; i0 += TRUNC_MAXP) {
    PolarBatch pb{};
    int nmax = 0;
    for (int i = i0; i < std::min(n, i0 + TRUNC_MAXP); ++i) {
      pb.a[pb.n++] = a[i];
      nmax = std::max(nmax, a[i].n);
    }
    if (nmax == 0) continue;
    k_polar_form<<<dim3(std::min(64, (nmax * nmax + 255) / 256), pb.n), 256, 0, s>>>(pb);
    ++launches;
  }
  return launches;
}

int launch_gather_rows(const GatherArgs* a, int n, cudaStream_t s) {
  int launches = 0;
  for (int i0 = 0; i0 < n; i0 += TRUNC_MAXP) {
    GatherBatch gb{};
    int chimax = 0;
    for (int i = i0; i < std::min(n, i0 + TRUNC_MAXP); ++i) {
      gb.a[gb.n++] = a[i];
      chimax = std::max(chimax, a[i].chi);
    }
    if (chimax == 0) continue;
    k_gather<<<dim3(chimax, gb.n), 256, 0, s>>>(gb);
    ++launches;
  }
  return launches;
}

int launch_init_product(double2* const* B, double* const* lam, const int* occ_dev, int L, int d, cudaStream_t s) {
  k_init_product<<<L, 32, 0, s>>>(B, lam, occ_dev, L, d);
  return 1;
}

int launch_densities(const DensityArgs* a, int n, cudaStream_t s) {
  int launches = 0;
  for (int i0 = 0; i0 < n; i0 += 32) {
    DensityBatch db{};
    for (int i = i0; i < std::min(n, i0 + 32); ++i) db.a[db.n++] = a[i];
    k_densities<<<db.n, 256, 0, s>>>(db);
    ++launches;
  }
  return launches;
}

__global__ void k_shift_pair(const double2* B, const double* lam, double2* out, int chl, int d, int chr, int shift,
                             int mode, int wd) {
  const long long total = (long long)chl * d * chr;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(e / ((long long)d * chr));
    const int s = (int)((e / chr) % d);
    const int c = (int)(e % chr);
    const int w = (mode == 1) ? s % wd : s / wd;
    double2 v = make_double2(0.0, 0.0);
    if (w < wd - 1 && s + shift < d) {
      const double f = (lam ? lam[a] * lam[a] : 1.0) * sqrt((double)(w + 1));
      const double2 x = B[((long long)a * d + s + shift) * chr + c];
      v = make_double2(f * x.x, f * x.y);
    }
    out[e] = v;
  }
}

__global__ void k_pair_hop(const double2* B, const double* lam, int chl, int d, int chr, int wd, double2* out) {
  __shared__ double sr[32], si[32];
  double re = 0.0, im = 0.0;
  const long long total = (long long)chl * d * chr;
  for (long long e = threadIdx.x; e < total; e += blockDim.x) {
    const int a = (int)(e / ((long long)d * chr));
    const int s = (int)((e / chr) % d);  // sigma' = s'_a wd + s'_b
    const int c = (int)(e % chr);
    const int sa = s / wd, sb = s % wd;
    if (sa >= wd - 1 || sb < 1) continue;
    const double f = lam[a] * lam[a] * sqrt((double)(sa + 1) * sb);
    const double2 x = B[e];                                          // B[a, sigma', b]
    const double2 y = B[((long long)a * d + s + wd - 1) * chr + c];  // B[a, (s'_a + 1, s'_b - 1), b]
    re = fma(f, y.x * x.x + y.y * x.y, re);                         // conj(y) x
    im = fma(f, y.x * x.y - y.y * x.x, im);
  }
  re = warp_sum(re);
  im = warp_sum(im);
  if ((threadIdx.x & 31) == 0) { sr[threadIdx.x >> 5] = re; si[threadIdx.x >> 5] = im; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0, m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { r += sr[w]; m += si[w]; }
    *out = make_double2(r, m);
  }
}

int launch_shift_pair(const double2* B, const double* lam, double2* out, int chl, int d, int chr, int shift, int mode,
                      int wd, cudaStream_t s) {
  k_shift_pair<<<grid_for((long long)chl * d * chr), 256, 0, s>>>(B, lam, out, chl, d, chr, shift, mode, wd);
  return 1;
}

int launch_pair_hop(const double2* B, const double* lam, int chl, int d, int chr, int wd, double2* out, cudaStream_t s) {
  k_pair_hop<<<1, 256, 0, s>>>(B, lam, chl, d, chr, wd, out);
  return 1;
}

int launch_shift_left(const double2* B, const double* lam, double2* out, int chl, int d, int chr, cudaStream_t s) {
  k_shift_left<<<grid_for((long long)chl * d * chr), 256, 0, s>>>(B, lam, out, chl, d, chr);
  return 1;
}

int launch_shift_right(const double2* B, double2* out, int chl, int d, int chr, cudaStream_t s) {
  k_shift_right<<<grid_for((long long)chl * d * chr), 256, 0, s>>>(B, out, chl, d, chr);
  return 1;
}

int launch_trace_product(const double2* X, const double2* Yt, int chi, double2* out, cudaStream_t s) {
  k_trace_product<<<1, 256, 0, s>>>(X, Yt, chi, out);
  return 1;
}

__global__ void k_graph_check_eig(const __grid_constant__ GraphEig g) {
  const int t = threadIdx.x;
  if (t == 0 && *g.bar_err != 0u) atomicOr(g.flag, 4);
  if (t >= g.n) return;
  const double tr = *g.trace[t];
  if (!(isfinite(tr) && tr > 0.0)) {
    atomicOr(g.flag, 1);
    return;
  }
  const double floor_v = g.floor_rel[t] * tr;
  if (!(g.evals[t][g.kmax[t] - 1] > floor_v)) atomicOr(g.flag, 2);
}

__global__ void k_graph_check_trunc(const __grid_constant__ GraphTrunc g) {
  const int t = threadIdx.x;
  if (t == 0 && *g.status != 0) atomicOr(g.flag, 16);
  if (t >= g.n) return;
  if (*g.chi[t] != g.expect[t]) atomicOr(g.flag, 8);
  *g.w_out[t] = *g.w[t];
}

__global__ void k_scale_inv(double2* X, long long n, const double* norm) {
  const double f = 1.0 / *norm;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double2 x = X[e];
    X[e] = make_double2(x.x * f, x.y * f);
  }
}

int launch_graph_check_eig(const GraphEig& g, cudaStream_t s) {
  k_graph_check_eig<<<1, 32, 0, s>>>(g);
  return 1;
}

int launch_graph_check_trunc(const GraphTrunc& g, cudaStream_t s) {
  k_graph_check_trunc<<<1, 32, 0, s>>>(g);
  return 1;
}

int launch_scale_inv(double2* X, long long n, const double* norm, cudaStream_t s) {
  if (n <= 0) return 0;
  k_scale_inv<<<grid_for(n), 256, 0, s>>>(X, n, norm);
  return 1;
}

int launch_check_finite(const double* x, int n, int* status, cudaStream_t s) {
  k_check_finite<<<grid_for(n), 256, 0, s>>>(x, n, status);
  return 1;
}

}  // namespace ptebd
