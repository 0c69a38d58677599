// Internal declarations shared by the library's translation units.
#pragma once

#include <complex>
#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

namespace ptebd {

// ---- host gate builder (gates_host.cpp) --------------------------------------
std::vector<std::complex<double>> three_site_term(int L, int n_max, double U, double J, double Jnnn,
                                                  double K, double jc, int j);
// max_sweeps: limit of the cyclic Jacobi eigen-solver (false if it did not converge).
bool build_gate(int L, int n_max, double U, double J, double Jnnn, double K, double jc, int j,
                double tau, std::vector<std::complex<double>>& G, int max_sweeps = 60);
// Super sites (pairs of physical sites): the term of super bond k (1-based) on the chain
// padded to even length, d^4 x d^4 over positions (2k-1, 2k, 2k+1, 2k+2), and its gate.
std::vector<std::complex<double>> supersite_bond_term(int L, int n_max, double U, double J, double Jnnn, double K,
                                                      double jc, int k);
bool build_gate_supersite(int L, int n_max, double U, double J, double Jnnn, double K, double jc, int k,
                          double tau, std::vector<std::complex<double>>& G, int max_sweeps = 60);

// ---- grouped GEMM (kernels_gemm.cu) ------------------------------------------
// C = alpha * op(A) * op(B) [+ C], op in {N, C = conjugate transpose, CJ = conjugate}; complex
// (double2) or real (double).  Up to GEMM_MAXP independent problems, each
// optionally strided-batched, share one launch.  Optional scalings:
//   s_red[k / red_div]  multiplies A(i, k) along the reduction index,
//   s_row[i / row_div], s_col[j / col_div] multiply the result.
enum { OP_N = 0, OP_C = 1, OP_CJ = 2 };  // CJ: element-wise conjugate, no transpose
constexpr int GEMM_MAXP = 16;

struct GemmProb {
  const void* A;
  const void* B;
  void* C;
  long long lda, ldb, ldc, sA, sB, sC;
  const double* s_red;
  const double* s_row;
  const double* s_col;
  double alpha_re, alpha_im;
  int M, N, K, batch;
  int red_div, row_div, col_div, accumulate;
  int herm;  // result is Hermitian (M == N, B = A^+): only lower tiles are computed, then mirrored
  const double* s_red_b;  // optional factor of B along the reduction index (red_div as s_red)
};

struct GemmBatch {
  GemmProb p[GEMM_MAXP];
  int tile_start[GEMM_MAXP + 1];
  int nprob, opA, opB, mixed;
};

// ---- complex GEMM as split 3xTF32 on tcgen05 tensor cores (kernels_tf32.cu) ------
// C = alpha * A * op(B), A complex M x K (op N), op(B) in {N, C}; FP64 complex in
// memory, FP32 accumulation in tensor memory.
struct TcGemmProb {
  const double2* A;
  const double2* B;
  double2* C;
  long long lda, ldb, ldc, sA, sB, sC;
  double alpha;
  int M, N, K, batch, opB;
};
constexpr int TC_MAXP = 24;
struct TcGemmBatch {
  TcGemmProb p[TC_MAXP];
  int tile_start[TC_MAXP + 1];
  int nprob;
  int* status;  // set to TEBD_ERR_TIMEOUT if a bounded wait runs out
};
int tc_gemm_launch(const std::vector<TcGemmProb>& probs, int* status, cudaStream_t s);

// ---- FP64-accurate complex GEMM on bf16 tensor cores, exact digit splitting (kernels_ozaki.cu)
// C[i][j] = alpha * s_row[i / row_div] * s_col[j / col_div] * sum_k a(i, k) b(j, k)
// with a(i, k) = op(X_a[i * rs + k * ks]) * scale[k / scale_div] (op: conj if set), b likewise.
struct OzOperand {
  const double2* X;
  long long rs, ks;
  const double* scale;  // optional factor along the reduction index
  int scale_div, conj;
  int real;  // X holds real doubles (element (r, k) = X_real[r * rs + k * ks], imaginary part 0)
};
struct OzProb {
  OzOperand a, b;  // b is ignored when gram is set
  int M, N, K;
  double2* C;
  long long ldc;
  double alpha;
  const double* s_row;
  const double* s_col;
  int row_div, col_div;
  int herm;  // Hermitian result (M == N): only j <= i is computed, then mirrored
  int gram;  // b(j, k) = conj(a(j, k)), N = M: the digits of a serve both operands
  int beta;  // 1: C += result (for herm, the lower triangle is read), 0: C = result
  double* Creal;  // if set, the real part of the result goes here (ldc in doubles) instead of C
  void* ws;  // oz_workspace_bytes(M, N, K, gram) bytes, 256-byte aligned, owned by the caller
};
constexpr int OZ_MAXP = 16;
struct OzPackJob {
  const double2* X;
  long long rs, ks;
  const double* scale;
  int scale_div, conj, rows, K, nrb, nkt, real;
  uint16_t* P0;  // digit plane written with form type0 (null: none)
  uint16_t* P1;
  int type0, type1;
  int* e;  // row exponents [nrb * 32]
};
struct OzPackBatch {
  OzPackJob job[2 * OZ_MAXP];
  int block_start[2 * OZ_MAXP + 1];
  int njob;
};
struct OzTile {
  const uint16_t* DA;
  const uint16_t* D1;
  const uint16_t* D2;
  const int* eA;
  const int* eB;
  double2* C;
  double* Creal;
  long long ldc;
  double alpha;
  const double* s_row;
  const double* s_col;
  int row_div, col_div, M, N, nkt, nrbA, nrbB, herm, tiles_n, beta;
};
struct OzGemmBatch {
  OzTile p[OZ_MAXP];
  int tile_start[OZ_MAXP + 1];
  int nprob;
  int* status;  // set to TEBD_ERR_TIMEOUT if a bounded wait runs out
};
size_t oz_workspace_bytes(int M, int N, int K, bool gram);
int oz_gemm_launch(const std::vector<OzProb>& probs, int* status, cudaStream_t s);

class Gemm {
 public:
  Gemm(bool complex_, int opA, int opB) : cplx_(complex_), opA_(opA), opB_(opB) {}
  GemmProb& add(int M, int N, int K, const void* A, long long lda, const void* B, long long ldb, void* C,
                long long ldc);
  // Launch everything added so far (in chunks of GEMM_MAXP) on stream; returns launches issued.
  // mixed: complex problems with op(A) = N, op(B) in {N, C}, real alpha and no
  // scalings run as split 3xTF32 on the tensor cores instead of FP64.
  int launch(cudaStream_t s, bool mixed = false, int* status = nullptr);
  size_t size() const { return probs_.size(); }

 private:
  bool cplx_;
  int opA_, opB_;
  std::vector<GemmProb> probs_;
};

// One problem, launched without any host or device allocation.
int gemm_launch_single(bool complex_, int opA, int opB, const GemmProb& p, cudaStream_t s);

// ---- eigen-solver for batches of Hermitian matrices (kernels_eig.cu) ---------
// Matrices per eigen-solver batch: one cooperative launch of the reduction serves them
// all, so its per-column grid barriers are paid once per batch (the blocked form
// decomposes hundreds of charge blocks per layer).
constexpr int EIG_MAXP = 64;
// Triples per batch of the dense form (its truncation and gather batches hold 24).
constexpr int CHUNK_MAXP = 24;

struct EigMat {
  double2* H;        // m x m Hermitian (full storage), row-major, ld = m; reflectors end in rows
  double* d;         // tridiagonal diagonal [m]
  double* e;         // sub-diagonal [m]
  double2* tau;      // Householder scalars [m]
  double2* part;     // partial dot products [EIG_PARTS], one per 32-column strip
  double2* p;        // p = tau A22 v [m]
  double* evals;     // eigenvalues, descending [kmax]
  double* trace;     // [1] trace of H (sum of Re H_rr), taken before reduction
  double* Z;         // m x K real eigenvectors of T (row-major, ld = K)
  double* Z2;        // m x K scratch (Newton-Schulz ping-pong)
  double* S;         // K x K scratch
  double* work;      // inverse-iteration LU scratch, 5 * m * K doubles
  double2* U;        // K x m eigenvectors of H, one per row (U[j*m + r] = u_j[r])
  double2* pan;      // panel arrays of the blocked reduction [eig_panel_doubles2(m)]
  int m, kmax, K;
};

struct EigBatch {
  EigMat a[EIG_MAXP];
  int n;
  unsigned int* bar;  // grid-barrier state {count, generation, error} for the persistent reduction
  long long wait_clocks;  // limit of each grid-barrier wait of the reduction (clock64 ticks)
  int panel_blocks;       // blocks per SM of the reduction's cooperative grid (0: as many as fit, at most 3)
};

constexpr int EIG_PARTS = 384;  // partial sums of p^+ v, one per strip of 32 columns (m <= 12288)

// Each returns the number of kernel launches issued.
int eig_trace(const EigBatch& b, cudaStream_t s);
// Blocked (panels of 32 columns): one cooperative launch per panel plus the
// trailing rank-64 update, on the exact-digit tensor-core engine when mixed
// (oz_ws[i]: a digit workspace per matrix) or the FP64 GEMM otherwise.
// Returns the launches issued, or -1 if a cooperative launch is refused.  A
// barrier that times out sets b.bar[2] (checked by the caller after synchronising).
int eig_tridiagonalize(const EigBatch& b, bool mixed, void* const* oz_ws, int* status, cudaStream_t s);
size_t eig_panel_doubles2(int m);  // complex elements of EigMat::pan for an m x m matrix
int eig_bisect(const EigBatch& b, cudaStream_t s);
// Eigenvalues needed per matrix of a cut (matrices whose spectra are merged): those at
// or above the cut's target-th largest eigenvalue and the floor floor_rel x the cut's
// trace, at most kmax.  The tridiagonal (d, e) and trace of every matrix are in place.
struct ThrCut {
  const EigMat* mats;  // device array of the cut's matrices
  int n, target;
  double floor_rel;
  int* kmax_out;       // device [n]
};
int eig_cut_counts(const ThrCut* cuts_dev, int ncuts, cudaStream_t s);
// Inverse iteration on T for eigenvalues 0..K-1, Newton-Schulz orthonormalisation,
// and back-transformation U = Q Z: in the mixed path in blocks of 64 reflectors
// (compact WY form, block products on the exact-digit engine), in the FP64 path
// reflector by reflector.
// Reads a[i].K (set from the eigenvalues).
int eig_vectors(const EigBatch& b, bool mixed, void* const* oz_ws, int* status, cudaStream_t s);

// ---- small kernels (kernels_misc.cu) -------------------------------------------
struct TruncArgs {
  const double2* Y;  // K x n rows u_k^+ theta'
  int K, n;
  const double* trace;
  double* s_sorted;   // [K] descending ||Y_k||
  int* perm;          // [K]
  double* lam_out;    // [chi'] s / ||s_kept||
  int* chi_out;       // [1]
  double* norm_out;   // [1] ||s_kept||
  double* w_out;      // [1] discarded weight of this truncation
  double* w_total;    // accumulated (device)
  int chi_max;
  double w_cut, eps_rel;
  int* status;        // device status word
};
constexpr int TRUNC_MAXP = 24;
struct TruncBatch {
  TruncArgs a[TRUNC_MAXP];
  int n;
};
int launch_truncate(const TruncBatch& b, cudaStream_t s);

struct GatherArgs {
  const double2* Y;
  const int* perm;
  const double* s_sorted;
  double2* out;  // chi x n
  int chi, n;
};
int launch_gather_rows(const GatherArgs* a, int n, cudaStream_t s);

// G <- 3/2 I - 1/2 G for square complex matrices (the Newton-Schulz polar step).
struct PolarArgs {
  double2* G;
  int n;
};
int launch_polar_form(const PolarArgs* a, int n, cudaStream_t s);

int launch_init_product(double2* const* B, double* const* lam, const int* occ_dev, int L, int d,
                        cudaStream_t s);

struct DensityArgs {
  const double2* B;
  const double* lam;
  double* out;
  int chl, d, chr;
  int wmode, wd;  // occupation of local state s: s (0), s / wd (1, first site of a pair), s % wd (2)
};
int launch_densities(const DensityArgs* a, int n, cudaStream_t s);

// P'[(a,s),c] = lam_a^2 sqrt(s+1) B[a,s+1,c] (s < d-1), 0 for s = d-1
int launch_shift_left(const double2* B, const double* lam, double2* out, int chl, int d, int chr,
                      cudaStream_t s);
// Q'[c,(t,b)] = sqrt(t+1) B[c,t+1,b] (t < d-1), 0 for t = d-1
int launch_shift_right(const double2* B, double2* out, int chl, int d, int chr, cudaStream_t s);
// out[(a,s),c] = f lam_a^2 sqrt(w(s)+1) B[a, s+shift, c] where w(s) < wd - 1, else 0, with
// w(s) = s % wd (mode 1) or s / wd (mode 2); f = 1 and lam optional (NULL: no lam^2).  The
// raising operator of one site of a super site (pairs of sites, sigma = s_a wd + s_b).
int launch_shift_pair(const double2* B, const double* lam, double2* out, int chl, int d, int chr, int shift, int mode,
                      int wd, cudaStream_t s);
// out = sum_{a,b} lam_a^2 sum_sigma' sqrt(s'_a + 1) sqrt(s'_b) conj(B[a, sigma' + wd - 1, b]) B[a, sigma', b]
// over s'_a < wd - 1, s'_b >= 1: <b+_(2k-1) b_(2k)> inside super site k.
int launch_pair_hop(const double2* B, const double* lam, int chl, int d, int chr, int wd, double2* out, cudaStream_t s);
// out = sum_{c,c'} X[c,c'] Yt[c',c]
int launch_trace_product(const double2* X, const double2* Yt, int chi, double2* out, cudaStream_t s);

int launch_check_finite(const double* x, int n, int* status, cudaStream_t s);

// ---- device-side checks of a captured step (CUDA-graph replay, api.cu) ------------------
constexpr int GRAPH_MAXT = 32;
// After the eigenvalues of a batch: each trace finite and positive, the kmax-th
// eigenvalue above floor_rel x trace (so the host would have asked for all kmax
// vectors), and no grid-barrier timeout.  Failed checks are OR-ed into *flag.
struct GraphEig {
  const double* evals[GRAPH_MAXT];
  const double* trace[GRAPH_MAXT];
  int kmax[GRAPH_MAXT];
  double floor_rel[GRAPH_MAXT];
  int n;
  const unsigned int* bar_err;
  int* flag;
};
int launch_graph_check_eig(const GraphEig& g, cudaStream_t s);
// After a truncation: chi' equal to the capacity the capture assumed, the truncation
// status clear; the discarded weight copied to w_out[i].
struct GraphTrunc {
  const int* chi[GRAPH_MAXT];
  int expect[GRAPH_MAXT];
  const double* w[GRAPH_MAXT];
  double* w_out[GRAPH_MAXT];
  int n;
  const int* status;
  int* flag;
};
int launch_graph_check_trunc(const GraphTrunc& g, cudaStream_t s);
// X[0..n) *= 1 / *norm (the renormalisation of a rebuilt site, norm on the device)
int launch_scale_inv(double2* X, long long n, const double* norm, cudaStream_t s);

}  // namespace ptebd
