// FP64 Hermitian eigen-solver for batches of Gram matrices H = theta' theta'^+.
//
// The truncated SVD of every local update (Sec. II B) is taken through the
// Gram matrix: its eigenvectors are the left singular vectors of theta'.
// Stages (each batched over all triples of a layer):
//   1. Householder reduction H = Q T Q^+ with T real symmetric tridiagonal
//      (reflectors H(k) = I - tau_k v_k v_k^+ with real beta_k, so the
//      sub-diagonal is real), blocked: one cooperative launch per panel of 32
//      columns plus a Hermitian rank-64 update of the trailing matrix.
//   2. Multisection on (division-free) Sturm counts for the kmax largest eigenvalues of T.
//   3. Inverse iteration for the K kept eigenvalues (one thread per
//      eigenvector, LU with partial pivoting of T - lambda I), with
//      Gram-Schmidt inside groups of nearly equal eigenvalues.
//   4. Newton-Schulz orthonormalisation Z <- Z (3I - Z^T Z)/2, three rounds.
//   5. Back-transformation U = Q Z: in blocks of 64 reflectors (compact WY
//      form) in the tensor-core paths, reflector by reflector with 8
//      eigenvectors per block in the FP64 path.
// All reductions use a fixed order, so results are bitwise reproducible.
#include "ptebd_internal.h"

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <vector>

namespace ptebd {

namespace {

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {  // a*b + c
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(-a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ double2 cfma_conj(double2 a, double2 b, double2 c) {  // conj(a)*b + c
  c.x = fma(a.x, b.x, c.x);
  c.x = fma(a.y, b.y, c.x);
  c.y = fma(a.x, b.y, c.y);
  c.y = fma(-a.y, b.x, c.y);
  return c;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return __shfl_sync(0xffffffffu, v, 0);
}
__device__ __forceinline__ double2 warp_sum2(double2 v) { return make_double2(warp_sum(v.x), warp_sum(v.y)); }

// Sum over the block (blockDim.x a multiple of 32, <= 1024); every thread gets the result.
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

__device__ double block_min(double v, double* sh) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = (l < nw) ? sh[l] : DBL_MAX;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmin(t, __shfl_xor_sync(0xffffffffu, t, o));
    if (l == 0) sh[32] = t;
  }
  __syncthreads();
  return sh[32];
}

constexpr int NT = 256;

// ---- trace --------------------------------------------------------------------
__global__ void k_trace(const __grid_constant__ EigBatch b) {
  const EigMat& M = b.a[blockIdx.x];
  __shared__ double sh[33];
  double s = 0.0;
  for (int r = threadIdx.x; r < M.m; r += blockDim.x) s += M.H[(size_t)r * M.m + r].x;
  s = block_sum(s, sh);
  if (threadIdx.x == 0) *M.trace = s;
}

// ---- bisection --------------------------------------------------------------------
// Number of eigenvalues of T below x: sign changes of the leading principal
// minors p_i = (d_i - x) p_{i-1} - e_{i-1}^2 p_{i-2} (Sturm's theorem), with
// a zero minor counted as a change.  Division-free: FP64 division is the
// slowest operation on this part, and the minors are kept in range by exact
// rescaling with 2^-500 / 2^500.  ee[i] = e_i^2 (k_esq).  The loop is bound by
// the FP64 pipe (two DFMA per clock per SM), so only the recurrence itself runs
// there: the zero, sign and range tests read the IEEE-754 fields with integer
// operations.  Rescaling by exact powers of two leaves every sign unchanged.
__device__ __forceinline__ int sturm_count(const double* d, const double* ee, int m, double x) {
  const double big = 0x1p500, small = 0x1p-500;
  double pm = 1.0, p = d[0] - x;
  if (p == 0.0) p = -small;
  long long bp = __double_as_longlong(p);
  int cnt = (int)((unsigned long long)bp >> 63);
  for (int i = 1; i < m; ++i) {
    double pn = fma(d[i] - x, p, -(ee[i - 1] * pm));
    long long bn = __double_as_longlong(pn);
    if ((bn << 1) == 0) {  // a zero minor takes the sign opposite to the previous one
      pn = (bp < 0) ? small : -small;
      bn = __double_as_longlong(pn);
    }
    cnt += (int)((unsigned long long)(bn ^ bp) >> 63);
    pm = p;
    p = pn;
    bp = bn;
    const int ex = (int)((bn >> 52) & 0x7FF);
    if (ex > 1023 + 500) { p *= small; pm *= small; bp = __double_as_longlong(p); }
    else if (ex < 1023 - 500) { p *= big; pm *= big; bp = __double_as_longlong(p); }
  }
  return cnt;
}

// ee[i] = e_i^2 of every tridiagonal, for the Sturm counts, in the inverse-iteration
// scratch (free until the eigenvectors are computed).
__global__ void k_esq(const __grid_constant__ EigBatch b) {
  const EigMat& M = b.a[blockIdx.y];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M.m; i += gridDim.x * blockDim.x)
    M.work[i] = (i < M.m - 1) ? M.e[i] * M.e[i] : 0.0;
}

__device__ void gershgorin(const double* d, const double* e, int m, double* sh, double& gl, double& gu) {
  double lo = DBL_MAX, hi = DBL_MAX;  // hi stored negated for a min-reduction
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    double r = 0.0;
    if (i > 0) r += fabs(e[i - 1]);
    if (i < m - 1) r += fabs(e[i]);
    lo = fmin(lo, d[i] - r);
    hi = fmin(hi, -(d[i] + r));
  }
  gl = block_min(lo, sh);
  gu = -block_min(hi, sh);
}

// Multisection with 4 points: a warp serves eight eigenvalues, four lanes each; per
// iteration the lanes of a group count the eigenvalues below 4 interior points of
// their interval, which shrinks it 5-fold (~23 iterations to machine precision).
// The counts are bound by the FP64 pipe once a batch holds many matrices (the
// blocked form's charge blocks): 4 points take 92 counts per eigenvalue against
// 136 with 8 points, at 1.35x the serial iterations.
__global__ void k_bisect(const __grid_constant__ EigBatch b) {
  const EigMat& M = b.a[blockIdx.y];
  const int m = M.m;
  __shared__ double sh[33];
  double gl, gu;
  gershgorin(M.d, M.e, m, sh, gl, gu);
  const int lane = threadIdx.x & 31, g = lane >> 2, sub = lane & 3;
  const int j = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 8 + g;
  const bool active = j < M.kmax && j < m;
  const double bnorm = fmax(fabs(gl), fabs(gu));
  const double eps = DBL_EPSILON, tiny = DBL_MIN * fmax(1.0, bnorm * bnorm);
  double lo = gl - 2.0 * eps * bnorm * m - 4.0 * tiny;
  double hi = gu + 2.0 * eps * bnorm * m + 4.0 * tiny;
  const double atol = 2.0 * eps * bnorm + 4.0 * tiny;
  const int target = m - 1 - j;  // ascending index of the j-th largest
  for (int it = 0; it < 64; ++it) {
    const bool conv = !(hi - lo > atol);
    if (__all_sync(0xffffffffu, conv || !active)) break;
    const double x = lo + (hi - lo) * (double)(sub + 1) * 0.2;
    const bool above = active && !conv && sturm_count(M.d, M.work, m, x) > target;  // eigenvalue below x
    const unsigned gb = (__ballot_sync(0xffffffffu, above) >> (4 * g)) & 0xFu;
    const int l0 = gb ? (__ffs(gb) - 1) : 4;  // first point above the eigenvalue (4: none)
    const double xa = __shfl_sync(0xffffffffu, x, 4 * g + (l0 > 0 ? l0 - 1 : 0));
    const double xb = __shfl_sync(0xffffffffu, x, 4 * g + (l0 < 4 ? l0 : 3));
    if (active && !conv) {
      if (l0 > 0) lo = xa;
      if (l0 < 4) hi = xb;
    }
  }
  if (active && sub == 0) M.evals[j] = 0.5 * (lo + hi);
}

// ---- eigenvalue counts of a cut -------------------------------------------------------
// A cut's spectrum is the union of its matrices' (the charge blocks of one truncated
// SVD).  Rule T keeps at most `target` values of the cut, so each matrix needs only
// its eigenvalues above the cut's target-th largest one (and above the floor
// floor_rel x the cut's trace).  One block per cut finds that threshold by
// multisection on the summed Sturm counts: P points per matrix per iteration, each
// iteration shrinking the bracket by P + 1, then writes per matrix the number of
// its eigenvalues at or above the bracket's lower end (capped by kmax).  The search
// ends early at a point whose count is exactly the target.  A cut's counts all run on
// one SM, whose FP64 pipe bounds them (every count is m dependent steps), so few
// points per iteration (P <= 7) do less work in total than a wide multisection.
__device__ __forceinline__ int count_at_or_above(const EigMat& M, double x) { return M.m - sturm_count(M.d, M.work, M.m, x); }

__global__ void __launch_bounds__(1024) k_cut_counts(const ThrCut* __restrict__ cuts) {
  const ThrCut C = cuts[blockIdx.x];
  __shared__ double sh[33];
  __shared__ int cnt[64];
  __shared__ double lo_sh, hi_sh;
  __shared__ int go_sh;
  // the cut's trace and an upper bound of its spectrum (Gershgorin)
  double tr = 0.0, up = 0.0;
  for (int i = threadIdx.x; i < C.n; i += blockDim.x) tr += *C.mats[i].trace;
  for (int i = 0; i < C.n; ++i) {
    const EigMat& M = C.mats[i];
    for (int r = threadIdx.x; r < M.m; r += blockDim.x) {
      double g = M.d[r];
      if (r > 0) g += fabs(M.e[r - 1]);
      if (r < M.m - 1) g += fabs(M.e[r]);
      up = fmax(up, g);
    }
  }
  tr = block_sum(tr, sh);
  up = -block_min(-up, sh);
  const double floor_v = C.floor_rel * tr;
  // how many eigenvalues lie at or above the floor
  if (threadIdx.x == 0) cnt[0] = 0;
  __syncthreads();
  {
    int mine = 0;
    for (int i = threadIdx.x; i < C.n; i += blockDim.x) mine += min(C.mats[i].kmax, count_at_or_above(C.mats[i], floor_v));
    atomicAdd(&cnt[0], mine);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    lo_sh = floor_v;
    hi_sh = fmax(up, floor_v) * (1.0 + 4.0 * DBL_EPSILON) + DBL_MIN;
    go_sh = cnt[0] > C.target;
  }
  __syncthreads();
  const int P = max(1, min(7, (int)blockDim.x / max(C.n, 1)));
  for (int it = 0; it < 80 && go_sh; ++it) {
    const double lo = lo_sh, hi = hi_sh;
    if (threadIdx.x < P) cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int pidx = threadIdx.x; pidx < C.n * P; pidx += blockDim.x) {
      const int i = pidx / P, j = pidx - i * P;
      const double x = lo + (hi - lo) * (double)(j + 1) / (double)(P + 1);
      atomicAdd(&cnt[j], min(C.mats[i].kmax, count_at_or_above(C.mats[i], x)));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int jb = -1;  // the last point still holding at least `target` values
      for (int j = 0; j < P; ++j)
        if (cnt[j] >= C.target) jb = j;
      const double nlo = (jb >= 0) ? lo + (hi - lo) * (double)(jb + 1) / (double)(P + 1) : lo;
      const double nhi = (jb + 1 < P) ? lo + (hi - lo) * (double)(jb + 2) / (double)(P + 1) : hi;
      lo_sh = nlo;
      hi_sh = nhi;
      go_sh = (jb < 0 || cnt[jb] != C.target) && (nhi - nlo) > 4.0 * DBL_EPSILON * fmax(fabs(nhi), DBL_MIN);
    }
    __syncthreads();
  }
  const double x = lo_sh;
  for (int i = threadIdx.x; i < C.n; i += blockDim.x)
    C.kmax_out[i] = min(C.mats[i].kmax, count_at_or_above(C.mats[i], x));
}

// ---- inverse iteration ----------------------------------------------------------------
__device__ __forceinline__ double hash_uniform(unsigned long long a, unsigned long long b) {
  unsigned long long z = a * 0x9E3779B97F4A7C15ull + b * 0xBF58476D1CE4E5B9ull + 0x94D049BB133111EBull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

// LU with partial pivoting of T - sigma I (tridiagonal; one fill-in diagonal).
// Row i of U: (u0, u1, u2) at columns (i, i+1, i+2); l = multiplier; piv = 1 if rows swapped.
__device__ void tri_lu(const double* d, const double* e, int m, double sigma, double tiny, double* U0, double* U1,
                       double* U2, double* Lm, double* Pv, int ld) {
  double u = d[0] - sigma, v = (m > 1) ? e[0] : 0.0, w = 0.0;
  for (int i = 0; i < m - 1; ++i) {
    const double c = e[i];                       // sub-diagonal entry of row i+1
    const double a = d[i + 1] - sigma;           // diagonal of row i+1
    const double bb = (i + 1 < m - 1) ? e[i + 1] : 0.0;  // super-diagonal of row i+1
    if (fabs(c) > fabs(u)) {
      const double l = u / c;
      U0[(size_t)i * ld] = c; U1[(size_t)i * ld] = a; U2[(size_t)i * ld] = bb;
      Lm[(size_t)i * ld] = l; Pv[(size_t)i * ld] = 1.0;
      const double nu = v - l * a, nv = w - l * bb;
      u = nu; v = nv; w = 0.0;
    } else {
      if (u == 0.0) u = tiny;
      const double l = c / u;
      U0[(size_t)i * ld] = u; U1[(size_t)i * ld] = v; U2[(size_t)i * ld] = w;
      Lm[(size_t)i * ld] = l; Pv[(size_t)i * ld] = 0.0;
      const double nu = a - l * v, nv = bb - l * w;
      u = nu; v = nv; w = 0.0;
    }
    if (fabs(U0[(size_t)i * ld]) < tiny) U0[(size_t)i * ld] = copysign(tiny, U0[(size_t)i * ld]);
  }
  if (fabs(u) < tiny) u = copysign(tiny, u);
  U0[(size_t)(m - 1) * ld] = u; U1[(size_t)(m - 1) * ld] = 0.0; U2[(size_t)(m - 1) * ld] = 0.0;
}

__device__ void tri_solve(int m, const double* U0, const double* U1, const double* U2, const double* Lm,
                          const double* Pv, int ld, double* z) {
  // forward: apply the row operations of the factorisation to z
  double cur = z[0];
  for (int i = 0; i < m - 1; ++i) {
    const double nxt = z[(size_t)(i + 1) * ld];
    const double l = Lm[(size_t)i * ld];
    if (Pv[(size_t)i * ld] != 0.0) {
      z[(size_t)i * ld] = nxt;
      cur = cur - l * nxt;
    } else {
      z[(size_t)i * ld] = cur;
      cur = nxt - l * cur;
    }
  }
  z[(size_t)(m - 1) * ld] = cur;
  // back substitution
  double z1 = 0.0, z2 = 0.0;  // z[i+1], z[i+2]
  for (int i = m - 1; i >= 0; --i) {
    const double zi = (z[(size_t)i * ld] - U1[(size_t)i * ld] * z1 - U2[(size_t)i * ld] * z2) / U0[(size_t)i * ld];
    z[(size_t)i * ld] = zi;
    z2 = z1;
    z1 = zi;
  }
}

__global__ void k_inviter(const __grid_constant__ EigBatch b) {
  const EigMat& M = b.a[blockIdx.y];
  const int m = M.m, K = M.K;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= K) return;
  const double* ev = M.evals;
  double tnorm = 0.0;
  for (int i = 0; i < m; ++i) {
    double r = fabs(M.d[i]);
    if (i > 0) r += fabs(M.e[i - 1]);
    if (i < m - 1) r += fabs(M.e[i]);
    tnorm = fmax(tnorm, r);
  }
  if (tnorm == 0.0) tnorm = 1.0;
  // Bisection places each shift within ~2 eps tnorm of its eigenvalue; eigenvalues
  // closer than 100x that are treated as one group and orthogonalised explicitly.
  const double gtol = 200.0 * DBL_EPSILON * tnorm;
  if (j > 0 && ev[j - 1] - ev[j] <= gtol) return;  // not the first of its group
  int g = j + 1;
  while (g < K && ev[g - 1] - ev[g] <= gtol) ++g;
  const double tiny = DBL_EPSILON * tnorm;
  const int ld = K;
  for (int q = j; q < g; ++q) {
    double* U0 = M.work + q;
    double* U1 = U0 + (size_t)m * K;
    double* U2 = U1 + (size_t)m * K;
    double* Lm = U2 + (size_t)m * K;
    double* Pv = Lm + (size_t)m * K;
    tri_lu(M.d, M.e, m, ev[q], tiny, U0, U1, U2, Lm, Pv, ld);
    double* z = M.Z + q;
    for (int i = 0; i < m; ++i) z[(size_t)i * ld] = hash_uniform(q + 1, i + 1);
    for (int it = 0; it < 3; ++it) {
      tri_solve(m, U0, U1, U2, Lm, Pv, ld, z);
      double mx = 0.0;
      for (int i = 0; i < m; ++i) mx = fmax(mx, fabs(z[(size_t)i * ld]));
      const double inv = (mx > 0.0) ? 1.0 / mx : 1.0;
      for (int i = 0; i < m; ++i) z[(size_t)i * ld] *= inv;
      for (int p = j; p < q; ++p) {  // Gram-Schmidt against earlier group members
        const double* y = M.Z + p;
        double dot = 0.0;
        for (int i = 0; i < m; ++i) dot = fma(y[(size_t)i * ld], z[(size_t)i * ld], dot);
        for (int i = 0; i < m; ++i) z[(size_t)i * ld] -= dot * y[(size_t)i * ld];
      }
      double nrm = 0.0;
      for (int i = 0; i < m; ++i) nrm = fma(z[(size_t)i * ld], z[(size_t)i * ld], nrm);
      nrm = sqrt(nrm);
      const double s = (nrm > 0.0) ? 1.0 / nrm : 0.0;
      for (int i = 0; i < m; ++i) z[(size_t)i * ld] *= s;
    }
  }
}

// S <- 1.5 I - 0.5 S
__global__ void k_ns_form(const __grid_constant__ EigBatch b) {
  const EigMat& M = b.a[blockIdx.y];
  const int K = M.K;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < K * K; idx += gridDim.x * blockDim.x) {
    const int r = idx / K, c = idx % K;
    M.S[idx] = (r == c ? 1.5 : 0.0) - 0.5 * M.S[idx];
  }
}

// U[j][r] = Z[r][j] (real -> complex, transposed).
__global__ void k_z_to_u(const __grid_constant__ EigBatch b, int use_z2) {
  const EigMat& M = b.a[blockIdx.z];
  const int m = M.m, K = M.K;
  __shared__ double tile[32][33];
  const double* Z = use_z2 ? M.Z2 : M.Z;
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  if (r0 >= m || c0 >= K) return;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < m && c < K) ? Z[(size_t)r * K + c] : 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (c < K && r < m) M.U[(size_t)c * m + r] = make_double2(tile[threadIdx.x][i], 0.0);
  }
}

constexpr int CPB = 8;  // eigenvectors per block in the back-transformation

// FP64 path: U <- H(0) H(1) ... H(m-2) U reflector by reflector, one block per CPB
// eigenvectors; per reflector the CPB dot products v^+ u are reduced together.
// (On FP64 CUDA cores this keeps more blocks busy than the blocked form's thin products.)
__global__ void __launch_bounds__(NT) k_backtransform(const __grid_constant__ EigBatch b) {
  const EigMat& M = b.a[blockIdx.y];
  const int m = M.m, K = M.K;
  const int c0 = blockIdx.x * CPB;
  if (c0 >= K) return;
  const int ncol = min(CPB, K - c0);
  __shared__ double2 red[NT / 32][CPB];
  __shared__ double2 wsh[CPB];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = m - 2; k >= 0; --k) {
    const double2 tau = M.tau[k];
    if (tau.x == 0.0 && tau.y == 0.0) continue;
    const int n = m - k - 1;
    const double2* v = M.H + (size_t)k * m + k + 1;
    double2 acc[CPB];
#pragma unroll
    for (int cc = 0; cc < CPB; ++cc) acc[cc] = make_double2(0.0, 0.0);
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
      const double2 vr = v[r];
#pragma unroll
      for (int cc = 0; cc < CPB; ++cc)
        if (cc < ncol) acc[cc] = cfma_conj(vr, M.U[(size_t)(c0 + cc) * m + k + 1 + r], acc[cc]);
    }
#pragma unroll
    for (int cc = 0; cc < CPB; ++cc) {
      const double2 t = warp_sum2(acc[cc]);
      if (lane == 0) red[warp][cc] = t;
    }
    __syncthreads();
    if (threadIdx.x < CPB) {
      double2 t = make_double2(0.0, 0.0);
      for (int w = 0; w < NT / 32; ++w) t = cadd(t, red[w][threadIdx.x]);
      wsh[threadIdx.x] = cmul(tau, t);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
      const double2 vr = v[r];
#pragma unroll
      for (int cc = 0; cc < CPB; ++cc) {
        if (cc < ncol) {
          double2* u = M.U + (size_t)(c0 + cc) * m + k + 1 + r;
          *u = csub(*u, cmul(vr, wsh[cc]));
        }
      }
    }
    __syncthreads();
  }
}

// ---- blocked back-transformation ----------------------------------------------------------
// U <- Q Z with Q = H(0) H(1) ... H(m-2) is applied as blocks of BT reflectors,
// Q_p = H(k0) ... H(k0+BT-1) = I - V T V^+ (compact WY form, T upper triangular:
// T[i][i] = tau_i, T[0:i, i] = -tau_i T[0:i, 0:i] (V^+ V)[0:i, i]), last block first:
// U^T <- U^T - V T (V^+ U^T), i.e. three matrix products per block on the rows of U.
constexpr int BT = 64;  // reflectors per block

// Trailing indices per slab of the reduction's Hermitian product.  A function of the matrix's
// own size, so its arithmetic could never depend on its batch; measured on GB300, 64-wide
// slabs for the blocked form's sizes (more items per column, more partial sums per strip)
// were slower than 256 at every size, so every matrix takes 256.
__host__ __device__ __forceinline__ int td_chunk(int) { return 256; }

__host__ __device__ inline size_t bt_offset(int m) {
  const size_t slabs = (size_t)((m + 31) / 32) * ((m + td_chunk(m) - 1) / td_chunk(m));
  return (size_t)m * 128 + (size_t)EIG_PARTS * 64 + slabs * 64;
}
// V (m x BT) and conj(V) reuse the panel arrays; then G = V^+ V, T^T, S = U conj(V), S T^T.
__device__ __forceinline__ double2* bt_V(const EigMat& M) { return M.pan; }
__device__ __forceinline__ double2* bt_Vc(const EigMat& M) { return M.pan + (size_t)M.m * BT; }
__device__ __forceinline__ double2* bt_G(const EigMat& M) { return M.pan + bt_offset(M.m); }
__device__ __forceinline__ double2* bt_Tt(const EigMat& M) { return bt_G(M) + BT * BT; }

// Column i of V = v_{k0+i} (unit entry at row k0+i+1, zero above), from the rows of H.
__global__ void k_bt_prep(const __grid_constant__ EigBatch b, int k0) {
  const EigMat& M = b.a[blockIdx.y];
  const int m = M.m;
  if (M.K == 0 || k0 >= m - 1) return;
  double2* V = bt_V(M);
  double2* Vc = bt_Vc(M);
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < m * BT; idx += gridDim.x * blockDim.x) {
    const int r = idx / BT, i = idx % BT, k = k0 + i;
    double2 v = make_double2(0.0, 0.0);
    if (k < m - 1) {
      if (r == k + 1) v = make_double2(1.0, 0.0);
      else if (r > k + 1) v = M.H[(size_t)k * m + r];
    }
    V[idx] = v;
    Vc[idx] = cconj(v);
  }
}

// T of the block from G = V^+ V and tau (one block per matrix; four threads per
// row of T share each column's sum), written transposed.
__global__ void __launch_bounds__(4 * BT) k_bt_T(const __grid_constant__ EigBatch b, int k0) {
  const EigMat& M = b.a[blockIdx.x];
  const int m = M.m;
  if (M.K == 0 || k0 >= m - 1) return;
  const int nb = min(BT, m - 1 - k0);
  extern __shared__ double2 Tsh[];  // BT x (BT + 1)
  const double2* G = bt_G(M);
  for (int idx = threadIdx.x; idx < BT * (BT + 1); idx += blockDim.x) Tsh[idx] = make_double2(0.0, 0.0);
  __syncthreads();
  const int l = threadIdx.x >> 2, part = threadIdx.x & 3;
  for (int i = 0; i < nb; ++i) {
    const double2 ti = M.tau[k0 + i];
    double2 acc = make_double2(0.0, 0.0);
    if (l < i)
      for (int q = l + part; q < i; q += 4) acc = cfma(Tsh[l * (BT + 1) + q], G[q * BT + i], acc);
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);
    if (part == 0) {
      if (l < i) Tsh[l * (BT + 1) + i] = make_double2(-(ti.x * acc.x - ti.y * acc.y), -(ti.x * acc.y + ti.y * acc.x));
      else if (l == i) Tsh[l * (BT + 1) + i] = ti;
    }
    __syncthreads();
  }
  double2* Tt = bt_Tt(M);
  for (int idx = threadIdx.x; idx < BT * BT; idx += blockDim.x) {
    const int r = idx / BT, c = idx % BT;  // Tt[r][c] = T[c][r]
    Tt[idx] = Tsh[c * (BT + 1) + r];
  }
}

// ---- blocked Householder reduction ---------------------------------------------------------
// Panels of TD_NB columns.  Within a panel the trailing matrix is left as it was
// at the panel start; each column's Hermitian product runs on that stored upper
// triangle (read once per column, as balanced slabs) and is corrected with the
// panel's earlier (v_i, w_i).  Only the next pivot row is brought up to date, by
// all blocks.  After the panel the trailing matrix takes the whole rank-2*TD_NB
// update as one Hermitian matrix product (tensor cores in the mixed path).  Every
// FP64 operation is scarce on this part, so sums stay in registers and every
// reduction has a fixed order (bitwise reproducible).  Three grid barriers per column.

constexpr int TD_THREADS = 256;
constexpr int TD_WARPS = TD_THREADS / 32;
constexpr int TD_STRIP = 32;
constexpr int TD_NB = 32;      // columns per panel of the blocked reduction
// A column whose largest off-diagonal entry lies below 2^-900 is taken as already
// reduced (tau = 0).  The Gram matrices here have trace ~1, so such entries are far
// below their rounding; they do arise, as rounding noise that each Gram product
// squares, in empty regions of the chain, and once subnormal the scale 1/amax of
// the reflector would overflow and turn the column into NaN.
constexpr double REFL_FLUSH = 0x1p-900;
// The last TD_TAIL or fewer columns of every matrix are reduced by one block per
// matrix with the trailing matrix in shared memory (k_tridiag_tail): there the
// cooperative kernel would pay three grid barriers per column for very little work.
// A matrix takes part in the panels k0 < tail_start(m) (a multiple of TD_NB), so the
// split depends on its own size only and each result is independent of its batch.
constexpr int TD_TAIL = 64;
__host__ __device__ __forceinline__ int tail_start(int m) {
  return m <= TD_TAIL ? 0 : ((m - TD_TAIL + TD_NB - 1) / TD_NB) * TD_NB;
}


// Grid barrier for a cooperative launch.  st = {arrival count, unused, error}.
// Every block adds 1 to the count with a fire-and-forget release reduction
// (no serialised round trips) and polls it with acquire loads until it reaches
// the next multiple of the grid size (`target`, advanced by each call).  Waits
// at most `limit` clocks (2e9, ~1 s, unless the handle's "wait_limit_clocks"
// says otherwise); on timeout it records the failure in st[2] and returns
// false so every block can leave.  The count starts at 0 per launch.
__device__ bool grid_sync(unsigned int* st, unsigned int& target, long long limit) {
  __shared__ int ok_sh;
  __syncthreads();
  target += gridDim.x;
  if (threadIdx.x == 0) {
    volatile unsigned int* verr = st + 2;
    int ok = 1;
    __threadfence();
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(st) : "memory");
    const long long t0 = clock64();
    while (true) {
      unsigned int v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(st) : "memory");
      if ((int)(v - target) >= 0) break;
      if (*verr) { ok = 0; break; }
      if (clock64() - t0 > limit) { atomicExch(st + 2, 1u); ok = 0; break; }
    }
    __threadfence();
    ok_sh = ok && (*verr == 0);
  }
  __syncthreads();
  return ok_sh != 0;
}

// Reflector of column k from row k by a whole block (block reductions).
__device__ void house_row_block(const EigMat& M, int k, double* sh, double2* scale_sh) {
  const int m = M.m;
  double2* row = M.H + (size_t)k * m;
  if (k == m - 1) {
    if (threadIdx.x == 0) {
      M.d[k] = row[k].x;
      M.e[k] = 0.0;
      M.tau[k] = make_double2(0.0, 0.0);
    }
    __syncthreads();
    return;
  }
  const int n = m - k - 1;
  double2* x = row + k + 1;
  double amax = 0.0;
  for (int r = threadIdx.x; r < n; r += blockDim.x) amax = fmax(amax, fmax(fabs(x[r].x), fabs(x[r].y)));
  amax = -block_min(-amax, sh);
  if (amax < REFL_FLUSH) amax = 0.0;
  const double sinv = (amax > 0.0) ? 1.0 / amax : 0.0;
  double s = 0.0;
  for (int r = 1 + threadIdx.x; r < n; r += blockDim.x) {
    const double vx = x[r].x * sinv, vy = x[r].y * sinv;
    s = fma(vx, vx, fma(vy, vy, s));
  }
  const double xnorm2 = block_sum(s, sh);
  if (threadIdx.x == 0) {
    const double ar = x[0].x * sinv, ai = -x[0].y * sinv;
    double beta;
    double2 tau, sc;
    if (amax == 0.0 || (xnorm2 == 0.0 && ai == 0.0)) {
      beta = x[0].x;
      tau = make_double2(0.0, 0.0);
      sc = make_double2(0.0, 0.0);
    } else {
      const double bs = -copysign(sqrt(ar * ar + ai * ai + xnorm2), ar);
      tau = make_double2((bs - ar) / bs, -ai / bs);
      const double zr = ar - bs, zi = ai, den = zr * zr + zi * zi;
      sc = make_double2(zr / den * sinv, -zi / den * sinv);
      beta = bs * amax;
    }
    M.d[k] = row[k].x;
    M.e[k] = beta;
    M.tau[k] = tau;
    *scale_sh = sc;
  }
  __syncthreads();
  const double2 sc = *scale_sh;
  for (int r = threadIdx.x; r < n; r += blockDim.x) x[r] = (r == 0) ? make_double2(1.0, 0.0) : cmul(cconj(x[r]), sc);
  __syncthreads();
}

// alpha = -tau (p^+ v) / 2 from the per-strip partial sums (fixed order): every
// warp forms the sum with its lanes striding the partials, so no thread runs a
// long dependent chain of loads.
__device__ __forceinline__ double2 rank2_alpha(const EigMat& M, int k, int n) {
  const int ns = (n + TD_STRIP - 1) / TD_STRIP;
  const int lane = threadIdx.x & 31;
  double2 dot = make_double2(0.0, 0.0);
  for (int j = lane; j < ns; j += 32) dot = cadd(dot, M.part[j]);
  dot = warp_sum2(dot);
  const double2 t2 = cmul(M.tau[k], dot);
  return make_double2(-0.5 * t2.x, -0.5 * t2.y);
}

// Panel arrays of a matrix: VW[r] = (v_0..v_{NB-1}, w_0..w_{NB-1})(r), WV[r] the
// same with the halves swapped (the second operand of the trailing update), the
// per-strip partial dots of the panel corrections, and the partial sums of the
// Hermitian product (64 per slab: column part, then row part).
__device__ __forceinline__ double2* pan_vw(const EigMat& M) { return M.pan; }
__device__ __forceinline__ double2* pan_wv(const EigMat& M) { return M.pan + (size_t)M.m * 2 * TD_NB; }
__device__ __forceinline__ double2* pan_xy(const EigMat& M) { return M.pan + (size_t)M.m * 4 * TD_NB; }
__device__ __forceinline__ double2* pan_hp(const EigMat& M) {
  return M.pan + (size_t)M.m * 4 * TD_NB + (size_t)EIG_PARTS * 2 * TD_NB;
}

// w = p + alpha v of column kp (panel index jp), stored as column jp of W.
__device__ void finish_w(const EigMat& M, int kp, int jp, double2 alpha) {
  const int m = M.m, n = m - kp - 1;
  if (n <= 0) return;
  const double2* v = M.H + (size_t)kp * m + kp + 1;
  double2* VW = pan_vw(M);
  double2* WV = pan_wv(M);
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const double2 w = cfma(alpha, v[r], M.p[r]);
    const size_t row = (size_t)(kp + 1 + r) * 2 * TD_NB;
    VW[row + TD_NB + jp] = w;
    WV[row + jp] = w;
  }
}


// Phase 1 of column k in one pass over row k held in registers (m - k <= 256 * P1_R):
// finish w of column k-1, the alpha part of the pivot row, and the reflector of
// column k (house_row_block's arithmetic: amax scaling, then the norm).
constexpr int P1_R = 8;
__device__ void phase1_regs(const EigMat& M, int k, int j, double* sh, double2* scale_sh) {
  const int m = M.m, nn = m - k;  // row k from the diagonal: element r <-> column k + r
  double2* row = M.H + (size_t)k * m;
  double2* VW = pan_vw(M);
  double2* WV = pan_wv(M);
  double2 a[P1_R];
  double amax = 0.0;
  if (j > 0) {
    const double2 alpha = rank2_alpha(M, k - 1, nn);
    const double2 sft = make_double2(M.p[0].x + 2.0 * alpha.x, M.p[0].y);
    const double2* vp = M.H + (size_t)(k - 1) * m + k;  // v_{k-1} from index k (vp[0] = 1)
#pragma unroll
    for (int u = 0; u < P1_R; ++u) {
      const int r = threadIdx.x + u * blockDim.x;
      a[u] = make_double2(0.0, 0.0);
      if (r < nn) {
        const double2 v = vp[r];
        const double2 w = cfma(alpha, v, M.p[r]);  // w_{k-1}(k + r)
        const size_t rw = (size_t)(k + r) * 2 * TD_NB;
        VW[rw + TD_NB + j - 1] = w;
        WV[rw + j - 1] = w;
        a[u] = csub(row[k + r], cmul(sft, cconj(v)));
        if (r >= 1) amax = fmax(amax, fmax(fabs(a[u].x), fabs(a[u].y)));
      }
    }
  } else {
#pragma unroll
    for (int u = 0; u < P1_R; ++u) {
      const int r = threadIdx.x + u * blockDim.x;
      a[u] = (r < nn) ? row[k + r] : make_double2(0.0, 0.0);
      if (r >= 1 && r < nn) amax = fmax(amax, fmax(fabs(a[u].x), fabs(a[u].y)));
    }
  }
  if (nn == 1) {  // last column: no reflector
    if (threadIdx.x == 0) {
      M.d[k] = a[0].x;
      M.e[k] = 0.0;
      M.tau[k] = make_double2(0.0, 0.0);
    }
    __syncthreads();
    return;
  }
  amax = -block_min(-amax, sh);
  if (amax < REFL_FLUSH) amax = 0.0;
  const double sinv = (amax > 0.0) ? 1.0 / amax : 0.0;
  double s2 = 0.0;
#pragma unroll
  for (int u = 0; u < P1_R; ++u) {
    const int r = threadIdx.x + u * blockDim.x;
    if (r >= 2 && r < nn) {
      const double vx = a[u].x * sinv, vy = a[u].y * sinv;
      s2 = fma(vx, vx, fma(vy, vy, s2));
    }
  }
  const double xnorm2 = block_sum(s2, sh);
  if (threadIdx.x == 1 % blockDim.x) {  // the thread holding r = 1 (x[0] of the reflector)
    const double2 x0 = a[0];
    const double ar = x0.x * sinv, ai = -x0.y * sinv;
    double beta;
    double2 tau, sc;
    if (amax == 0.0 || (xnorm2 == 0.0 && ai == 0.0)) {
      beta = x0.x;
      tau = make_double2(0.0, 0.0);
      sc = make_double2(0.0, 0.0);
    } else {
      const double bs = -copysign(sqrt(ar * ar + ai * ai + xnorm2), ar);
      tau = make_double2((bs - ar) / bs, -ai / bs);
      const double zr = ar - bs, zi = ai, den = zr * zr + zi * zi;
      sc = make_double2(zr / den * sinv, -zi / den * sinv);
      beta = bs * amax;
    }
    M.e[k] = beta;
    M.tau[k] = tau;
    *scale_sh = sc;
  }
  if (threadIdx.x == 0) M.d[k] = a[0].x;
  __syncthreads();
  const double2 sc = *scale_sh;
#pragma unroll
  for (int u = 0; u < P1_R; ++u) {
    const int r = threadIdx.x + u * blockDim.x;
    if (r < nn) {
      double2 out = a[u];  // r = 0: the diagonal element
      if (r >= 1) {
        out = (r == 1) ? make_double2(1.0, 0.0) : cmul(cconj(a[u]), sc);
        const size_t rw = (size_t)(k + r) * 2 * TD_NB;
        VW[rw + j] = out;
        WV[rw + TD_NB + j] = out;
      }
      row[k + r] = out;
    }
  }
  __syncthreads();
}

// Blocked Householder tridiagonalisation, one panel of columns [k0, k1) per
// cooperative launch (the trailing matrix from k0 on is current when it starts).
// Column k (panel index j) is reduced against A(k) = A(k0) - sum_{i<j} (v_i w_i^+ +
// w_i v_i^+) without forming A(k):
//   phase 1 (a block per matrix): w of column k-1 and the last term of row k (see
//           phase 3); the reflector of column k (v_k, tau_k).
//   phase 2 (slabs of 32 x td_chunk(m)): h = A(k0) v over the stored upper triangle,
//           and per-strip partials of w_i^+ v and v_i^+ v.
//   phase 3 (strips of 32): p = tau (h - sum_i (v_i (w_i^+ v) + w_i (v_i^+ v))), the
//           strip partials of p^+ v for alpha, and row k+1 brought to A(k+1) except
//           for the part of column k's own term that needs alpha.
// After the panel, the caller applies A -= V W^+ + W V^+ to rows and columns >= k1
// as one Hermitian rank-2*NB matrix product.
// Three blocks per SM (80 registers, a 64-byte spill): the reduction is latency bound
// (barrier and scoreboard stalls), so the extra resident warps hide part of it.
__global__ void __launch_bounds__(TD_THREADS, 3) k_tridiag_panel(const __grid_constant__ EigBatch b, int k0, int k1) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ double2 acc_sh[TD_WARPS][TD_STRIP];
  __shared__ double2 xy_sh[2 * TD_NB];
  __shared__ double2 vk_sh[2 * TD_NB];
  __shared__ double2 pv_sh[TD_WARPS][TD_STRIP];
  __shared__ double2 rv_sh[TD_WARPS][TD_STRIP];
  __shared__ double red_sh[33];
  __shared__ double2 scale_sh;
  __shared__ int pre2[EIG_MAXP + 1], pre3[EIG_MAXP + 1];  // items of phase 2 / 3 before each matrix
  unsigned int target = 0;  // barrier count expected at the next grid_sync
  for (int k = k0; k < k1; ++k) {
    const int j = k - k0;
    // ---- phase 1 (row k in registers when it fits, else in memory passes)
    for (int mi = blockIdx.x; mi < b.n; mi += gridDim.x) {
      const EigMat& M = b.a[mi];
      const int m = M.m;
      if (k >= tail_start(m)) continue;
      if (m - k <= P1_R * (int)blockDim.x) {
        phase1_regs(M, k, j, red_sh, &scale_sh);
        continue;
      }
      double2* row = M.H + (size_t)k * m;
      if (j > 0) {
        // Row k was brought to A(k) in phase 3 of column k-1 except for the alpha
        // part of that column's own term: with v_{k-1}(k) = 1 and w = p + alpha v it
        // is (p(k) + 2 Re alpha) conj(v_{k-1}(c)).
        const double2 alpha = rank2_alpha(M, k - 1, m - k);
        finish_w(M, k - 1, j - 1, alpha);
        const double2 sft = make_double2(M.p[0].x + 2.0 * alpha.x, M.p[0].y);
        const double2* vp = M.H + (size_t)(k - 1) * m;
        for (int c = k + threadIdx.x; c < m; c += blockDim.x) row[c] = csub(row[c], cmul(sft, cconj(vp[c])));
      }
      __syncthreads();
      house_row_block(M, k, red_sh, &scale_sh);
      double2* VWm = pan_vw(M);
      double2* WVm = pan_wv(M);
      for (int r = k + 1 + threadIdx.x; r < m; r += blockDim.x) {
        const double2 v = row[r];
        VWm[(size_t)r * 2 * TD_NB + j] = v;
        WVm[(size_t)r * 2 * TD_NB + TD_NB + j] = v;
      }
    }
    if (!grid_sync(b.bar, target, b.wait_clocks)) return;
    // ---- phase 2: h = A(k0) v by slabs.  Item (s, q) covers strip s (32 columns) and
    // chunk q (td_chunk(m) indices) of the trailing set: the column part reads the stored
    // rows r in chunk q above the strip's columns (r <= c, used as conj(A[r][c]) v[r]),
    // the row part reads the strip's rows at columns c > row in chunk q.  Every item
    // holds about 32 x chunk elements, so the work balances across blocks.  The items
    // before each matrix are counted once per column (pre2, pre3) and an item finds its
    // matrix by binary search.
    if (threadIdx.x < b.n) {  // items of each matrix, then their prefix sums
      const int i = threadIdx.x;
      const int n = (k < tail_start(b.a[i].m)) ? b.a[i].m - k - 1 : 0;
      const int ch = td_chunk(b.a[i].m);
      pre2[i + 1] = (n > 0) ? ((n + TD_STRIP - 1) / TD_STRIP) * ((n + ch - 1) / ch) : 0;
      pre3[i + 1] = (n > 0) ? (n + TD_STRIP - 1) / TD_STRIP : 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      pre2[0] = pre3[0] = 0;
      for (int i = 1; i <= b.n; ++i) {
        pre2[i] += pre2[i - 1];
        pre3[i] += pre3[i - 1];
      }
    }
    __syncthreads();
    for (int item = blockIdx.x; item < pre2[b.n]; item += gridDim.x) {
      int lo = 0, hi = b.n - 1;  // the last matrix whose first item is <= item
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre2[mid] <= item) lo = mid; else hi = mid - 1;
      }
      const int mi = lo, rem = item - pre2[mi];
      const EigMat& M = b.a[mi];
      const int m = M.m, n = m - k - 1, ch = td_chunk(m);
      const int nq = (n + ch - 1) / ch;
      const int sidx = rem / nq, q = rem % nq;
      const int c0 = sidx * TD_STRIP, w = min(TD_STRIP, n - c0);
      const int q0 = q * ch, q1 = min(n, q0 + ch);
      const double2* v = M.H + (size_t)k * m + k + 1;
      const double2* A = M.H + (size_t)(k + 1) * m + k + 1;
      const int c = c0 + lane;
      double2 acc = make_double2(0.0, 0.0);
      const int rend = min(q1, c0 + w);
      for (int r0 = q0 + warp; r0 < rend; r0 += 4 * TD_WARPS) {
        double2 a[4], vv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int r = r0 + u * TD_WARPS;
          const bool ok = r < rend && lane < w && c >= r;
          a[u] = ok ? A[(size_t)r * m + c] : make_double2(0.0, 0.0);
          vv[u] = r < rend ? v[r] : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) acc = cfma_conj(a[u], vv[u], acc);
      }
      acc_sh[warp][lane] = acc;
      for (int qq = warp; qq < TD_STRIP; qq += TD_WARPS) {
        double2 a2[4] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0), make_double2(0.0, 0.0),
                         make_double2(0.0, 0.0)};
        if (qq < w) {
          const int cc = c0 + qq;
          const double2* rowc = A + (size_t)cc * m;
          for (int r0 = max(q0, cc + 1) + lane; r0 < q1; r0 += 128) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int r = r0 + 32 * u;
              if (r < q1) a2[u] = cfma(rowc[r], v[r], a2[u]);
            }
          }
        }
        const double2 a2s = warp_sum2(cadd(cadd(a2[0], a2[1]), cadd(a2[2], a2[3])));
        if (lane == 0) pv_sh[0][qq] = a2s;
      }
      __syncthreads();
      if (warp == 0) {
        double2 p1 = make_double2(0.0, 0.0);
        for (int wq = 0; wq < TD_WARPS; ++wq) p1 = cadd(p1, acc_sh[wq][lane]);
        double2* hp = pan_hp(M) + (size_t)rem * 2 * TD_STRIP;
        hp[lane] = p1;
        hp[TD_STRIP + lane] = pv_sh[0][lane];
      }
      // partial dots of the panel corrections over this strip: w_i^+ v, v_i^+ v
      if (q == 0 && threadIdx.x < 2 * j) {
        const int i = threadIdx.x < j ? threadIdx.x : threadIdx.x - j;
        const int col = threadIdx.x < j ? TD_NB + i : i;  // w_i first, then v_i
        const double2* VW = pan_vw(M);
        double2 t = make_double2(0.0, 0.0);
        for (int qq = 0; qq < w; ++qq) t = cfma_conj(VW[(size_t)(k + 1 + c0 + qq) * 2 * TD_NB + col], v[c0 + qq], t);
        pan_xy(M)[(size_t)sidx * 2 * TD_NB + threadIdx.x] = t;
      }
      __syncthreads();
    }
    if (!grid_sync(b.bar, target, b.wait_clocks)) return;
    // ---- phase 3: corrections, tau, the strip partials of p^+ v, and row k+1
    for (int item = blockIdx.x; item < pre3[b.n]; item += gridDim.x) {
      int lo = 0, hi = b.n - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre3[mid] <= item) lo = mid; else hi = mid - 1;
      }
      const int mi = lo, rem = item - pre3[mi];
      const EigMat& M = b.a[mi];
      const int m = M.m, n = m - k - 1, ch = td_chunk(m);
      const int ns = (n + TD_STRIP - 1) / TD_STRIP;
      const int nq = (n + ch - 1) / ch;
      const int c0 = rem * TD_STRIP, w = min(TD_STRIP, n - c0);
      const double2* v = M.H + (size_t)k * m + k + 1;
      // Row k+1 (the next pivot, if it is in this panel) is brought to A(k+1) here,
      // spread over the strips, except for the alpha part of column k's term.
      const bool nextrow = (k + 1 < k1);
      if (threadIdx.x < 2 * j) {  // X_i = w_i^+ v, Y_i = v_i^+ v over the whole trailing set
        const double2* xy = pan_xy(M);
        double2 t = make_double2(0.0, 0.0);
#pragma unroll 4
        for (int s2 = 0; s2 < ns; ++s2) t = cadd(t, xy[(size_t)s2 * 2 * TD_NB + threadIdx.x]);
        xy_sh[threadIdx.x] = t;
        if (nextrow) {  // v_i(k+1) then w_i(k+1)
          const int i = threadIdx.x < j ? threadIdx.x : TD_NB + threadIdx.x - j;
          vk_sh[threadIdx.x] = pan_vw(M)[(size_t)(k + 1) * 2 * TD_NB + i];
        }
      }
      __syncthreads();
      // warp wq adds the terms i = wq, wq + 8, ... for the 32 elements of the strip
      double2 corr = make_double2(0.0, 0.0), rcorr = make_double2(0.0, 0.0);
      if (lane < w) {
        const double2* rc = pan_vw(M) + (size_t)(k + 1 + c0 + lane) * 2 * TD_NB;
        for (int i = warp; i < j; i += TD_WARPS) {
          const double2 vc = rc[i], wc = rc[TD_NB + i];
          corr = cfma(vc, xy_sh[i], corr);      // v_i(c) (w_i^+ v)
          corr = cfma(wc, xy_sh[j + i], corr);  // w_i(c) (v_i^+ v)
          if (nextrow) {                        // v_i(k+1) conj(w_i(c)) + w_i(k+1) conj(v_i(c))
            rcorr = cfma(vk_sh[i], cconj(wc), rcorr);
            rcorr = cfma(vk_sh[j + i], cconj(vc), rcorr);
          }
        }
      }
      pv_sh[warp][lane] = corr;
      rv_sh[warp][lane] = rcorr;
      __syncthreads();
      if (warp == 0) {
        double2 pd = make_double2(0.0, 0.0);
        if (lane < w) {
          double2 cs = make_double2(0.0, 0.0), rs = make_double2(0.0, 0.0);
          for (int wq = 0; wq < TD_WARPS; ++wq) {
            cs = cadd(cs, pv_sh[wq][lane]);
            rs = cadd(rs, rv_sh[wq][lane]);
          }
          const double2* hp = pan_hp(M) + (size_t)rem * nq * 2 * TD_STRIP;
          double2 h = make_double2(0.0, 0.0);
          for (int q = 0; q < nq; ++q)
            h = cadd(h, cadd(hp[(size_t)q * 2 * TD_STRIP + lane], hp[(size_t)q * 2 * TD_STRIP + TD_STRIP + lane]));
          const double2 pc = cmul(M.tau[k], csub(h, cs));
          M.p[c0 + lane] = pc;
          pd = cfma_conj(pc, v[c0 + lane], make_double2(0.0, 0.0));
          if (nextrow) {  // column k's term without alpha: conj(p(c)) (v_k(k+1) = 1)
            double2* a = M.H + (size_t)(k + 1) * m + k + 1 + c0 + lane;
            *a = csub(csub(*a, rs), cconj(pc));
          }
        }
        pd = warp_sum2(pd);
        if (lane == 0) M.part[rem] = pd;
      }
      __syncthreads();
    }
    if (!grid_sync(b.bar, target, b.wait_clocks)) return;
  }
  // w of the panel's last column
  for (int mi = blockIdx.x; mi < b.n; mi += gridDim.x) {
    const EigMat& M = b.a[mi];
    if (k0 < tail_start(M.m) && k1 - 1 < M.m - 1) finish_w(M, k1 - 1, k1 - 1 - k0, rank2_alpha(M, k1 - 1, M.m - k1));
  }
}

// The columns [tail_start(m), m) of one matrix per block, unblocked, with the
// trailing matrix (n <= TD_TAIL, current when the kernel starts) in shared memory
// as a full Hermitian matrix.  The reflectors are those of the panel kernel
// (phase1_regs' arithmetic on the pivot row), stored the same way in the rows of H;
// each column then applies A <- A - v w^+ - w v^+ with p = tau A v,
// w = p - (tau (p^+ v) / 2) v.  One fixed order per reduction.
constexpr int TL_LD = TD_TAIL + 1;
__global__ void __launch_bounds__(256) k_tridiag_tail(const __grid_constant__ EigBatch b) {
  extern __shared__ double2 tl_sh[];
  double2* As = tl_sh;                      // TD_TAIL x TL_LD
  double2* vs = As + TD_TAIL * TL_LD;       // v of the current column
  double2* ws = vs + TD_TAIL;               // p, then w
  __shared__ double red_sh[33];
  __shared__ double2 sc_sh, alpha_sh;
  const EigMat& M = b.a[blockIdx.x];
  const int m = M.m, k0 = tail_start(m), nt = m - k0;
  if (nt <= 0) return;
  for (int e = threadIdx.x; e < nt * nt; e += blockDim.x) {
    const int r = e / nt, c = e % nt;
    if (c >= r) {
      const double2 x = M.H[(size_t)(k0 + r) * m + k0 + c];
      As[r * TL_LD + c] = x;
      As[c * TL_LD + r] = cconj(x);
    }
  }
  __syncthreads();
  for (int j = 0; j < nt; ++j) {
    const int k = k0 + j, nn = nt - j;  // row j of the current matrix from its diagonal: nn entries
    const double2* row = As + j * TL_LD + j;
    if (nn == 1) {
      if (threadIdx.x == 0) {
        M.d[k] = row[0].x;
        M.e[k] = 0.0;
        M.tau[k] = make_double2(0.0, 0.0);
        M.H[(size_t)k * m + k] = row[0];
      }
      break;
    }
    double amax = 0.0;
    for (int r = 1 + threadIdx.x; r < nn; r += blockDim.x) amax = fmax(amax, fmax(fabs(row[r].x), fabs(row[r].y)));
    amax = -block_min(-amax, red_sh);
    if (amax < REFL_FLUSH) amax = 0.0;
    const double sinv = (amax > 0.0) ? 1.0 / amax : 0.0;
    double s2 = 0.0;
    for (int r = 2 + threadIdx.x; r < nn; r += blockDim.x) {
      const double vx = row[r].x * sinv, vy = row[r].y * sinv;
      s2 = fma(vx, vx, fma(vy, vy, s2));
    }
    const double xnorm2 = block_sum(s2, red_sh);
    if (threadIdx.x == 0) {
      const double2 x0 = row[1];
      const double ar = x0.x * sinv, ai = -x0.y * sinv;
      double beta;
      double2 tau, sc;
      if (amax == 0.0 || (xnorm2 == 0.0 && ai == 0.0)) {
        beta = x0.x;
        tau = make_double2(0.0, 0.0);
        sc = make_double2(0.0, 0.0);
      } else {
        const double bs = -copysign(sqrt(ar * ar + ai * ai + xnorm2), ar);
        tau = make_double2((bs - ar) / bs, -ai / bs);
        const double zr = ar - bs, zi = ai, den = zr * zr + zi * zi;
        sc = make_double2(zr / den * sinv, -zi / den * sinv);
        beta = bs * amax;
      }
      M.d[k] = row[0].x;
      M.e[k] = beta;
      M.tau[k] = tau;
      M.H[(size_t)k * m + k] = row[0];
      sc_sh = sc;
    }
    __syncthreads();
    const double2 sc = sc_sh, tau = M.tau[k];
    const int n = nn - 1;  // trailing indices r = 0..n-1 <-> rows/columns j+1+r
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
      const double2 v = (r == 0) ? make_double2(1.0, 0.0) : cmul(cconj(row[1 + r]), sc);
      vs[r] = v;
      M.H[(size_t)k * m + k + 1 + r] = v;
    }
    __syncthreads();
    // p = tau A v over the trailing block, four threads per row
    const double2* At = As + (j + 1) * TL_LD + (j + 1);
    {
      const int r = threadIdx.x >> 2, part = threadIdx.x & 3;
      double2 acc = make_double2(0.0, 0.0);
      if (r < n)
        for (int c = part; c < n; c += 4) acc = cfma(At[r * TL_LD + c], vs[c], acc);
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);
      if (part == 0 && r < n) ws[r] = cmul(tau, acc);
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // alpha = -tau (p^+ v) / 2
      double2 dot = make_double2(0.0, 0.0);
      for (int r = threadIdx.x; r < n; r += 32) dot = cfma_conj(ws[r], vs[r], dot);
      dot = warp_sum2(dot);
      if (threadIdx.x == 0) {
        const double2 t2 = cmul(tau, dot);
        alpha_sh = make_double2(-0.5 * t2.x, -0.5 * t2.y);
      }
    }
    __syncthreads();
    const double2 alpha = alpha_sh;
    for (int r = threadIdx.x; r < n; r += blockDim.x) ws[r] = cfma(alpha, vs[r], ws[r]);
    __syncthreads();
    double2* Aw = As + (j + 1) * TL_LD + (j + 1);
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int r = e / n, c = e % n;
      double2 a = Aw[r * TL_LD + c];
      a = csub(a, cmul(vs[r], cconj(ws[c])));
      a = csub(a, cmul(ws[r], cconj(vs[c])));
      Aw[r * TL_LD + c] = a;
    }
    __syncthreads();
  }
}

int max_m(const EigBatch& b) {
  int mm = 0;
  for (int i = 0; i < b.n; ++i) mm = std::max(mm, b.a[i].m);
  return mm;
}

}  // namespace

static_assert(sizeof(EigBatch) < 32000, "kernel parameter block too large (32 KB on sm_70 and later)");

int eig_trace(const EigBatch& b, cudaStream_t s) {
  if (b.n == 0) return 0;
  k_trace<<<b.n, NT, 0, s>>>(b);
  return 1;
}

int eig_tridiagonalize(const EigBatch& b, bool mixed, void* const* oz_ws, int* status, cudaStream_t s) {
  if (b.n == 0) return 0;
  const int mm = max_m(b);
  static int sms = 0, per_sm = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tridiag_panel, TD_THREADS, 0);
  }
  const int grid = std::max(1, sms * std::min(per_sm, b.panel_blocks > 0 ? b.panel_blocks : 3));
  int launches = 0;
  int kend = 0;  // panels run while any matrix has columns before its tail
  for (int i = 0; i < b.n; ++i) kend = std::max(kend, tail_start(b.a[i].m));
  for (int k0 = 0; k0 < kend; k0 += TD_NB) {
    int k1 = std::min(mm, k0 + TD_NB);
    // grid sized to the panel's largest phase (its first column's slabs): small matrices
    // get a small grid, whose barriers are cheaper; at least one block per active matrix
    long long items = 0;
    int active = 0;
    for (int i = 0; i < b.n; ++i) {
      if (k0 >= tail_start(b.a[i].m)) continue;
      ++active;
      const int n = b.a[i].m - k0 - 1;
      const int ch = td_chunk(b.a[i].m);
      if (n > 0) items += (long long)((n + TD_STRIP - 1) / TD_STRIP) * ((n + ch - 1) / ch);
    }
    const int gsz = (int)std::min<long long>(grid, std::max<long long>(active, items));
    cudaMemsetAsync(b.bar, 0, sizeof(unsigned int), s);  // arrival count of the grid barrier
    void* args[] = {const_cast<EigBatch*>(&b), &k0, &k1};
    if (cudaLaunchCooperativeKernel((const void*)k_tridiag_panel, dim3(gsz), dim3(TD_THREADS), args, 0, s) !=
        cudaSuccess)
      return -1;
    ++launches;
    // trailing update A[k1:, k1:] -= V W^+ + W V^+ (Hermitian, lower tiles mirrored)
    Gemm g(true, OP_N, OP_C);
    std::vector<OzProb> oz;
    for (int i = 0; i < b.n; ++i) {
      const EigMat& M = b.a[i];
      const int n = M.m - k1;
      if (n <= 0 || k0 >= tail_start(M.m)) continue;
      double2* C = M.H + (size_t)k1 * M.m + k1;
      const double2* VW = M.pan + (size_t)k1 * 2 * TD_NB;
      const double2* WV = M.pan + (size_t)M.m * 2 * TD_NB + (size_t)k1 * 2 * TD_NB;
      if (mixed) {
        OzProb q{};
        q.a = OzOperand{VW, 2 * TD_NB, 1, nullptr, 1, 0};
        q.b = OzOperand{WV, 2 * TD_NB, 1, nullptr, 1, 1};
        q.M = q.N = n;
        q.K = 2 * TD_NB;
        q.C = C;
        q.ldc = M.m;
        q.alpha = -1.0;
        q.beta = 1;
        q.row_div = q.col_div = 1;
        q.herm = 1;
        q.ws = oz_ws[i];
        oz.push_back(q);
      } else {
        GemmProb& p = g.add(n, n, 2 * TD_NB, VW, 2 * TD_NB, WV, 2 * TD_NB, C, M.m);
        p.alpha_re = -1.0;
        p.accumulate = 1;
        p.herm = 1;
      }
    }
    launches += mixed ? oz_gemm_launch(oz, status, s) : g.launch(s);
  }
  {
    constexpr int TL_SMEM = (TD_TAIL * TL_LD + 2 * TD_TAIL) * (int)sizeof(double2);
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_tridiag_tail, cudaFuncAttributeMaxDynamicSharedMemorySize, TL_SMEM);
      attr = true;
    }
    k_tridiag_tail<<<b.n, 256, TL_SMEM, s>>>(b);
    ++launches;
  }
  k_esq<<<dim3(std::max(1, std::min(64, (mm + 255) / 256)), b.n), 256, 0, s>>>(b);
  return launches + 1;
}

size_t eig_panel_doubles2(int m) {
  // panel arrays, then the back-transformation's G, T^T, S and S T^T
  return bt_offset(m) + 2 * BT * BT + (size_t)2 * m * BT;
}
static_assert(BT == 2 * TD_NB && TD_STRIP == 32, "bt_offset() mirrors the panel layout");

int eig_cut_counts(const ThrCut* cuts_dev, int ncuts, cudaStream_t s) {
  if (ncuts <= 0) return 0;
  k_cut_counts<<<ncuts, 1024, 0, s>>>(cuts_dev);
  return 1;
}

int eig_bisect(const EigBatch& b, cudaStream_t s) {
  if (b.n == 0) return 0;
  int km = 0;
  for (int i = 0; i < b.n; ++i) km = std::max(km, std::min(b.a[i].kmax, b.a[i].m));
  if (km == 0) return 0;
  k_bisect<<<dim3((km + 31) / 32, b.n), 128, 0, s>>>(b);  // four warps, eight eigenvalues each
  return 1;
}

int eig_vectors(const EigBatch& b0, bool mixed, void* const* oz_ws, int* status, cudaStream_t s) {
  if (b0.n == 0) return 0;
  EigBatch b = b0;
  int Kmax = 0, launches = 0;
  for (int i = 0; i < b.n; ++i) Kmax = std::max(Kmax, b.a[i].K);
  if (Kmax == 0) return 0;
  k_inviter<<<dim3((Kmax + 31) / 32, b.n), 32, 0, s>>>(b);
  ++launches;
  // Newton-Schulz: Z <- Z (1.5 I - 0.5 Z^T Z)
  bool in_z2 = false;
  for (int it = 0; it < 3; ++it) {
    Gemm g1(false, OP_C, OP_N), g2(false, OP_N, OP_N);
    std::vector<OzProb> o1, o2;  // the mixed path: the same real products on the exact-digit engine
    for (int i = 0; i < b.n; ++i) {
      const EigMat& M = b.a[i];
      if (M.K == 0) continue;
      const double* Zc = in_z2 ? M.Z2 : M.Z;
      double* Zn = in_z2 ? M.Z : M.Z2;
      if (mixed) {
        OzProb q{};
        q.row_div = q.col_div = 1;
        q.alpha = 1.0;
        q.ws = oz_ws[i];
        OzProb g = q;  // S = Z^T Z
        g.a = OzOperand{reinterpret_cast<const double2*>(Zc), 1, M.K, nullptr, 1, 0, 1};
        g.M = g.N = M.K; g.K = M.m; g.Creal = M.S; g.ldc = M.K; g.gram = g.herm = 1;
        o1.push_back(g);
        OzProb z = q;  // Z' = Z S
        z.a = OzOperand{reinterpret_cast<const double2*>(Zc), M.K, 1, nullptr, 1, 0, 1};
        z.b = OzOperand{reinterpret_cast<const double2*>(M.S), 1, M.K, nullptr, 1, 0, 1};
        z.M = M.m; z.N = M.K; z.K = M.K; z.Creal = Zn; z.ldc = M.K;
        o2.push_back(z);
      } else {
        g1.add(M.K, M.K, M.m, Zc, M.K, Zc, M.K, M.S, M.K);
      }
    }
    launches += mixed ? oz_gemm_launch(o1, status, s) : g1.launch(s);
    k_ns_form<<<dim3(std::max(1, std::min(64, (Kmax * Kmax + 255) / 256)), b.n), 256, 0, s>>>(b);
    ++launches;
    if (mixed) {
      launches += oz_gemm_launch(o2, status, s);
    } else {
      for (int i = 0; i < b.n; ++i) {
        const EigMat& M = b.a[i];
        if (M.K == 0) continue;
        const double* Zc = in_z2 ? M.Z2 : M.Z;
        double* Zn = in_z2 ? M.Z : M.Z2;
        g2.add(M.m, M.K, M.K, Zc, M.K, M.S, M.K, Zn, M.K);
      }
      launches += g2.launch(s);
    }
    in_z2 = !in_z2;
  }
  const int mm = max_m(b);
  k_z_to_u<<<dim3((mm + 31) / 32, (Kmax + 31) / 32, b.n), dim3(32, 8), 0, s>>>(b, in_z2 ? 1 : 0);
  ++launches;
  if (!mixed) {
    k_backtransform<<<dim3((Kmax + CPB - 1) / CPB, b.n), NT, 0, s>>>(b);
    return launches + 1;
  }
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_bt_T, cudaFuncAttributeMaxDynamicSharedMemorySize, BT * (BT + 1) * 16);
    attr = true;
  }
  const int nblk = (mm - 1 + BT - 1) / BT;
  for (int p = nblk - 1; p >= 0; --p) {
    const int k0 = p * BT;
    k_bt_prep<<<dim3(64, b.n), 256, 0, s>>>(b, k0);
    ++launches;
    std::vector<OzProb> oG, oS, oS2, oU;
    Gemm gG(true, OP_C, OP_N), gS(true, OP_N, OP_CJ), gS2(true, OP_N, OP_N), gU(true, OP_N, OP_C);
    for (int i = 0; i < b.n; ++i) {
      const EigMat& M = b.a[i];
      const int m = M.m, K = M.K, mr = m - k0 - 1;
      if (K == 0 || mr <= 0) continue;
      const double2* V = M.pan + (size_t)(k0 + 1) * BT;
      const double2* Vc = M.pan + (size_t)m * BT + (size_t)(k0 + 1) * BT;
      double2* G = M.pan + bt_offset(m);
      double2* Tt = G + BT * BT;
      double2* S = Tt + BT * BT;
      double2* S2 = S + (size_t)m * BT;
      double2* U = M.U + k0 + 1;
      if (mixed) {
        OzProb q{};
        q.row_div = q.col_div = 1;
        q.alpha = 1.0;
        q.ws = oz_ws[i];
        OzProb g = q;  // G = V^+ V
        g.a = OzOperand{V, 1, BT, nullptr, 1, 1};
        g.M = g.N = BT; g.K = mr; g.C = G; g.ldc = BT; g.gram = g.herm = 1;
        oG.push_back(g);
        OzProb t = q;  // S = U conj(V): S[j][i] = sum_r U[j][r] conj(V[r][i])
        t.a = OzOperand{U, m, 1, nullptr, 1, 0};
        t.b = OzOperand{V, 1, BT, nullptr, 1, 1};
        t.M = K; t.N = BT; t.K = mr; t.C = S; t.ldc = BT;
        oS.push_back(t);
        OzProb t2 = q;  // S2 = S T^T
        t2.a = OzOperand{S, BT, 1, nullptr, 1, 0};
        t2.b = OzOperand{Tt, 1, BT, nullptr, 1, 0};
        t2.M = K; t2.N = BT; t2.K = BT; t2.C = S2; t2.ldc = BT;
        oS2.push_back(t2);
        OzProb u = q;  // U -= S2 V^T
        u.a = OzOperand{S2, BT, 1, nullptr, 1, 0};
        u.b = OzOperand{V, BT, 1, nullptr, 1, 0};
        u.M = K; u.N = mr; u.K = BT; u.C = U; u.ldc = m; u.alpha = -1.0; u.beta = 1;
        oU.push_back(u);
      } else {
        gG.add(BT, BT, mr, V, BT, V, BT, G, BT);
        gS.add(K, BT, mr, U, m, V, BT, S, BT);
        gS2.add(K, BT, BT, S, BT, Tt, BT, S2, BT);
        GemmProb& pu = gU.add(K, mr, BT, S2, BT, Vc, BT, U, m);
        pu.alpha_re = -1.0;
        pu.accumulate = 1;
      }
    }
    launches += mixed ? oz_gemm_launch(oG, status, s) : gG.launch(s);
    k_bt_T<<<b.n, 4 * BT, BT * (BT + 1) * 16, s>>>(b, k0);
    ++launches;
    launches += mixed ? oz_gemm_launch(oS, status, s) : gS.launch(s);
    launches += mixed ? oz_gemm_launch(oS2, status, s) : gS2.launch(s);
    launches += mixed ? oz_gemm_launch(oU, status, s) : gU.launch(s);
  }
  return launches;
}

}  // namespace ptebd
