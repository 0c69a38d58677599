/*
 * ptebd.h - C ABI of the GB300 three-site TEBD library (libptebd.so).
 *
 * The library evolves a matrix product state in Vidal Gamma-lambda form
 * (stored as B_j = Gamma_j lambda_j, right canonical) under a second-order
 * Trotter split of the Bose-Hubbard chain with NN hopping J, NNN hopping
 * J_NNN, on-site U and a harmonic trap K about j_c (arXiv:2401.05301,
 * eq. (1)).  Each Trotter layer applies three-site gates exp(-i h_j tau) to
 * all triples (j, j+1, j+2) with the same j mod 3 at once; every local update
 * contracts theta, applies the gate, takes two truncated SVDs and rebuilds
 * B and lambda (Sec. II B).  Densities n_j (eq. (8)) and currents
 * 2 J Im <b+_j b_{j+1}> (eq. (5)) are measured from the canonical form.
 *
 * Conventions for every call:
 *   - Sites are 1-based in the physics (j = 1..L, j_c in the same coordinate);
 *     arrays passed across this ABI are 0-based C arrays over j = 1..L.
 *   - Time is in units of hbar/J (the paper's Sec. I A sets J = hbar = 1).
 *   - Every call returns a status (TEBD_OK = 0 or a negative TEBD_ERR_*),
 *     never throws, and never keeps a pointer the caller passed in.
 *   - All device memory is allocated and owned by the library, at
 *     tebd_create (state, gates) and at the first tebd_step (workspace).
 *   - A CUDA error puts the handle into a sticky error state: every later call
 *     except tebd_destroy / tebd_strerror returns TEBD_ERR_CUDA.
 *   - A handle is not thread safe; one handle issues work on one stream.
 */
#ifndef PTEBD_H
#define PTEBD_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tebd_ctx* tebd_handle;

/* Source of the Gaussian test matrices of the randomized truncation (option
 * "randomized"): called on the host once per truncated SVD with its index
 * `call` (0, 1, 2, ... in the order of the updates: layer by layer, triples in
 * increasing site order, cut 1 then cut 2 of each), its column count n and
 * sketch size l; fills out[2 n l] with the n x l complex matrix (row-major,
 * interleaved).  The random numbers are an input of the method. */
typedef void (*tebd_test_matrix_fn)(long long call, int n, int l, double* out, void* ctx);

enum {
  TEBD_OK = 0,
  TEBD_ERR_ARG = -1,           /* invalid argument (range, NULL, non-finite) */
  TEBD_ERR_OOM = -2,           /* device allocation failed */
  TEBD_ERR_CUDA = -3,          /* CUDA runtime error (sticky) */
  TEBD_ERR_STATE = -4,         /* call out of order (e.g. step before init) */
  TEBD_ERR_NOT_CONVERGED = -5, /* eigen-solver iteration limit reached */
  TEBD_ERR_TIMEOUT = -6,       /* bounded device wait ran out */
  TEBD_ERR_NONFINITE = -7,     /* NaN/Inf found in singular values */
  TEBD_ERR_TOO_LARGE = -8      /* size beyond a fixed capacity (tebd_bond_correlator_noalloc) */
};

/* Create a simulation of eq. (1) on L sites.
 *   L >= 3 (three-site gates), 1 <= n_max <= 7 (local dimension d = n_max+1),
 *   chi_max >= 1 (bond-dimension cap), U, J, J_NNN, K, j_c, dt finite, dt > 0.
 * Builds the (L-2) x 2 gates exp(-i h_j tau), tau in {dt/2, dt}, on the host
 * in FP64 (h_j: the three-site share of eq. (1), see tebd_gate_host), uploads
 * them, and allocates the MPS on the current CUDA device.  The state is
 * undefined until tebd_init_product.  *out receives the handle (NULL on error). */
int tebd_create(int L, int n_max, int chi_max, double U, double J, double J_NNN, double K,
                double j_c, double dt, tebd_handle* out);

/* Create a simulation of eq. (1) on L physical sites in the paper's own scheme
 * (Sec. II B): every two neighbouring sites form one super site of local dimension
 * d_e = (n_max + 1)^2 (basis sigma = s_a (n_max + 1) + s_b, s_a the left site), an
 * odd chain first gets one extra empty site at its end, so the MPS has
 * L_e = ceil(L / 2) super sites and nearest-neighbour two-site gates of dimension
 * d_e^2.  The super bond (k, k+1) holds the NN and both NNN hops between the two
 * super sites; each term inside a super site (its hop and on-site terms) is shared
 * equally among the one or two super bonds that contain it, so the bond terms sum
 * to eq. (1) on the padded chain.  Gates exp(-i h_k tau) are built per occupation
 * block (every term conserves N).  A step is odd bonds dt/2, even bonds dt, odd
 * bonds dt/2, one SVD per gate, the B-form two-site update.
 *   L >= 3, 1 <= n_max <= 4 (d_e <= 25), chi_max >= 1; other arguments as tebd_create.
 * On the handle: tebd_init_product takes the L physical occupations (the padded
 * site starts empty); tebd_set_state, tebd_get_site and tebd_bond_dims see the
 * L_e super sites; tebd_measure writes 2 L_e densities and 2 L_e - 1 currents of
 * the padded physical chain; tebd_layer takes residue 0 (odd bonds k = 1, 3, ...)
 * or 1 (even bonds).  "u1", "randomized" and trotter_order 4 are refused
 * (TEBD_ERR_ARG); a batch must not mix super-site and three-site handles. */
int tebd_create_supersite(int L, int n_max, int chi_max, double U, double J, double J_NNN, double K,
                          double j_c, double dt, tebd_handle* out);

/* Set a numerical option; valid before or between steps.
 *   "w_cut"   discarded-weight cut: keep the fewest values whose discarded
 *             weight sum_{i>chi'} p_i <= w_cut, p_i = s_i^2 / sum s^2  (default 0)
 *   "eps_rel" drop every value with p_i <= eps_rel (default 1e-12, the paper's eps)
 *   "precision" 0 = FP64 on the CUDA cores everywhere (default);
 *             1 = mixed: theta/gate/rebuild contractions as split 3xTF32 on the
 *             tensor cores (FP32 accumulation), the SVD stage FP64-accurate (its
 *             dense products as exact-digit bf16 tensor-core products);
 *             2 = FP64-accurate throughout: the contractions too as exact-digit
 *             tensor-core products (the small gate product on FP64 CUDA cores)
 *   "max_slots" cap on triples processed concurrently (0 = automatic)
 *   "randomized" 0 (default); 1: each truncated SVD of the dense form by the
 *             randomized range finder the paper points to (Sec. V; Halko, Martinsson
 *             and Tropp): a sketch of l = min(chi_max + "oversample", m, n) columns
 *             from a caller-supplied test matrix (tebd_set_test_matrices), "power_iters"
 *             re-orthonormalised power iterations, then the exact decomposition of the
 *             l x n matrix Q^+ theta'; rule T with the tail from ||theta'||_F^2.  Every
 *             product runs on the path's engine (exact-digit tensor-core products for
 *             precision 1 and 2).  Dense form only (TEBD_ERR_ARG with "u1").
 *   "oversample" p >= 0 (default 10), "power_iters" q >= 0 (default 2)
 *   "u1"      0 (default): dense local updates; 1: the particle-number blocked
 *             form of Sec. II B's U(1)-symmetric tensors.  Every gate conserves
 *             N, so each Schmidt vector carries a charge (tebd_set_charges) and
 *             the contractions and both truncated SVDs run block by block over
 *             the charges; rule T is applied to the merged spectrum of all blocks
 *             of a cut, and the kept vectors are stored sorted by charge.  The
 *             site tensors stay dense in device memory (zero outside their
 *             blocks), so measurement and state I/O are unchanged.  Valid before
 *             the first step only (TEBD_ERR_STATE afterwards).
 *   "trotter_order" 2 (default): the symmetric step A(dt/2) B(dt/2) C(dt) B(dt/2)
 *             A(dt/2); 4: Suzuki's fourth-order composition of that step,
 *             S2(p dt)^2 S2((1-4p) dt) S2(p dt)^2 with p = 1/(4 - 4^(1/3)) (25 layers;
 *             the cross-check of Appendix A).  Changing it rebuilds the gate table
 *             (four time arguments instead of two) and synchronises the stream.
 *   "jacobi_max_sweeps" sweep limit (1..1000, default 60) of the host Jacobi
 *             eigen-solver that exponentiates the three-site terms; changing it
 *             rebuilds the gate table, and a gate that does not converge within
 *             the limit makes the call return TEBD_ERR_NOT_CONVERGED (sticky).
 *   "graph"   0 (default); 1: replay whole steps as CUDA graphs where that is exact
 *             (dense three-site form; not with "u1", "randomized", super sites or
 *             "profile").  While every bond is at its capacity min(chi_max, d^...) the
 *             host's decisions after each truncation are known in advance (all kmax
 *             eigenvectors, chi' = capacity), so the second consecutive step of the same
 *             set of handles (tebd_step, or tebd_batch_step driven by hs[0]) is captured
 *             with those decisions checked on the device, and later steps replay it.  A
 *             replay whose checks fail (a truncation below capacity, a vector count the
 *             eps floor would have cut, a non-finite trace, a status) is undone from the
 *             state backup the graph takes first and the step runs the ordinary way, so
 *             results are bitwise those of the ordinary path.  A handle on the legacy
 *             default stream gets its own blocking stream.  Changing any option or the
 *             state makes the next step capture again.  (An addition: the paper's runs
 *             are not launch bound.)
 *   "graph_test_fallback" n >= 0 (diagnostic): treat the next n accepted replays as
 *             failed checks (state restored from the backup, step run the ordinary way),
 *             to test that path; unlike every other option it keeps the cached graph.
 *   "panel_blocks" 0 (default: as many as fit, at most 3) or 1..3: blocks per SM of the
 *             tridiagonal reduction's cooperative grid (a launch shape; the arithmetic and
 *             its order do not depend on it).  Chosen per (chi, d) bucket by the package's
 *             autotuner (paper_2401_05301_gb300/autotune.py).
 *   "wait_limit_clocks" limit, in GPU clock ticks (default 2e9, about 1 s), of
 *             every grid-barrier wait of the cooperative tridiagonal reduction.
 *             A wait that runs out records the failure, every block of the
 *             launch leaves, and the step returns TEBD_ERR_TIMEOUT (sticky); the
 *             CUDA context stays usable.  A diagnostic for the failure path: any
 *             limit far below the default makes a step fail.  (The mbarrier waits
 *             of the tensor-core kernels keep their fixed ~1 s limit, since one of
 *             them guards the release of tensor memory.)
 * Unknown key or out-of-range value: TEBD_ERR_ARG. */
int tebd_set_option(tebd_handle h, const char* key, double value);

/* Issue all work on the given cudaStream_t (NULL = legacy default stream).
 * The stream must belong to the handle's device and outlive its use.
 * Infrastructure: the paper has no counterpart. */
int tebd_set_stream(tebd_handle h, void* cuda_stream);

/* Reset the state to the product state |occ[0], ..., occ[L-1]> (eq. (2) form),
 * 0 <= occ[j] <= n_max; resets t, the step counter and w_total.  occ is a host
 * array of L ints, read before the call returns. */
int tebd_init_product(tebd_handle h, const int* occ);

/* Apply n_steps >= 0 full second-order steps A(dt/2) B(dt/2) C(dt) B(dt/2) A(dt/2),
 * where layer A holds the triples j = 1 mod 3, B: j = 2 mod 3, C: j = 0 mod 3.
 * Work is enqueued on the handle's stream; the call returns after the last
 * truncation decision of the last layer has been read back (the host needs
 * the new bond dimensions to size the next launches). */
int tebd_step(tebd_handle h, int n_steps);

/* Serving infrastructure (no counterpart in the paper): device bytes a handle
 * with these sizes holds once stepped and measured
 * (state, gates, workspace for min(triples per layer, 24, max_slots > 0 ?
 * max_slots : 24) concurrent local updates, measurement buffers; precision 1
 * and 2 add the digit planes of the exact-digit products),
 * written to *bytes.  Host-only arithmetic: used to admit simulations by an
 * HBM budget before creating them.  precision must be 0, 1 or 2.  The gate
 * table is counted for trotter_order 2 (order 4 holds twice as many gates). */
int tebd_estimate_bytes(int L, int n_max, int chi_max, int max_slots, int precision, double* bytes);

/* tebd_estimate_bytes for a handle of the particle-number-blocked form (option
 * "u1"): dense site tensors, gates and their occupation blocks, per workspace slot
 * an arena allowance for a saturated local update, and the exact-digit workspace
 * rings (the blocked arenas grow with the charge blocks; both allowances are fixed
 * multiples of the dense theta, 16 chi_max^2 d^3 bytes, fitted to the measured
 * footprint of a saturated chi = 1024, d = 5 state with 4, 8 and 21 slots).
 * Host-only arithmetic.  Serving infrastructure (no counterpart in the paper). */
int tebd_estimate_bytes_u1(int L, int n_max, int chi_max, int max_slots, int precision, double* bytes);

/* Batched form (an addition: the paper runs one chain per job, Sec. II B, IV):
 * advance n distinct handles (simulations with any L, n_max,
 * chi_max and parameters) by n_steps full steps together.  Within every
 * layer, the triples of all simulations are processed as shared batches: each
 * stage of the local update is one grouped launch over all of them.  Work
 * runs on hs[0]'s stream; all handles must be on the same device, hold a
 * state and use the same "precision" and "trotter_order" (else TEBD_ERR_ARG).  Each simulation's
 * result is bitwise the same as stepping it alone.  A device error marks every
 * member sticky. */
int tebd_batch_step(tebd_handle* hs, int n, int n_steps);

/* Apply one layer of the second-order split of Sec. II B only: every triple
 * j = residue + 1 (mod 3), 1-based
 * (residue in {0, 1, 2}), with tau = dt/2 (full = 0) or dt (full = 1).  The
 * step counter and t are unchanged.  Used to compare single layers of large
 * states against a reference.  Needs trotter_order 2 (else TEBD_ERR_ARG). */
int tebd_layer(tebd_handle h, int residue, int full);

/* Measure n_j (j = 1..L) into n_out[L] and current_j = 2 J Im <b+_j b_{j+1}>
 * (j = 1..L-1, positive = flow from j to j+1) into cur_out[L-1], both host
 * arrays of doubles owned by the caller.  Either pointer may be NULL to skip
 * it.  Synchronises the handle's stream. */
int tebd_measure(tebd_handle h, double* n_out, double* cur_out);

/* Serving infrastructure (no counterpart in the paper): the device bytes the
 * handle holds now (state, gates, workspace, measurement buffers, and the
 * blocked form's arenas, which grow to the high-water mark of its charge
 * blocks), written to *bytes. */
int tebd_device_bytes(tebd_handle h, double* bytes);

/* Current time t = steps * dt, accumulated discarded weight w_total
 * (sum of w over every truncation, Appendix B), and the largest bond
 * dimension.  Any pointer may be NULL. */
int tebd_stats(tebd_handle h, double* t, double* w_total, int* max_chi);

/* Copy the bond dimensions chi_k, k = 0..L (chi_0 = chi_L = 1), into chi[L+1]:
 * the MPS bond dimensions, capped by chi_max (Sec. II B). */
int tebd_bond_dims(tebd_handle h, int* chi);

/* Read back the B-form tensor B_k = Gamma_k lambda_k of Vidal's form (named in
 * Sec. I) for site k (0-based) as B[chi_k][d][chi_{k+1}] (complex FP64, real and
 * imaginary interleaved: 2 * chi_k * d * chi_{k+1} doubles) and/or the bond
 * vector lambda_k (chi_k doubles, k = 0..L).  Host buffers owned by the caller,
 * sized from tebd_bond_dims; either pointer may be NULL. */
int tebd_get_site(tebd_handle h, int k, double* B, double* lam);

/* Install a state: site tensors B_k (host, interleaved complex, shape
 * chi[k] x d x chi[k+1]) and bond vectors lam_k (host, chi[k] doubles,
 * k = 0..L), with chi[0] = chi[L] = 1 and chi[k] <= min(chi_max, d^k, d^(L-k)).
 * B_ptrs has L entries, lam_ptrs has L+1.  Resets t, steps and w_total.
 * Used to start from a saturated state.  The state is taken as given: the
 * method assumes the B-form of a normalised state (each B_k right-canonical,
 * sum_a lam_{k,a}^2 = 1), as a product state is and as each step keeps it up to
 * its truncation; the eigen-solver treats Gram entries below 2^-900 as zero,
 * which is far below rounding only for such a state. */
int tebd_set_state(tebd_handle h, const int* chi, const double* const* B_ptrs,
                   const double* const* lam_ptrs);

/* Bond charges for the particle-number (U(1)) blocked form of the option "u1"
 * (the paper's U(1)-symmetric tensors, Sec. II B).  q_ptrs has L+1 entries;
 * q_ptrs[k] is a host array of chi_k ints (chi from tebd_bond_dims): for each
 * Schmidt index of bond k, the number of bosons on the sites left of the bond.
 * Each array must be non-decreasing (every charge one contiguous run of the
 * index), 0 <= q <= n_max k, and q_ptrs[0][0] = 0.  The installed state must
 * vanish outside its blocks, B_k[a, s, b] = 0 unless q_{k+1}[b] = q_k[a] + s:
 * the blocked update reads only those blocks.  tebd_init_product sets the
 * charges of its product state itself; tebd_set_state clears them, and a
 * blocked step without them returns TEBD_ERR_STATE.  Arrays are read before
 * the call returns. */
int tebd_set_charges(tebd_handle h, const int* const* q_ptrs);

/* Install the test-matrix source of the randomized truncation (fn NULL removes
 * it) and restart its call index at 0.  ctx is passed to fn unchanged.  A
 * randomized step without a source returns TEBD_ERR_STATE; a source that
 * writes a non-finite value makes the step return TEBD_ERR_ARG.
 * Infrastructure for the method's random input (no counterpart in the paper). */
int tebd_set_test_matrices(tebd_handle h, tebd_test_matrix_fn fn, void* ctx);

/* Copy the charges of bond k (0 <= k <= L) into q[chi_k] (host).  After every
 * blocked local update the new bonds are sorted by charge.  TEBD_ERR_STATE if
 * the handle has no charges (after tebd_set_state without tebd_set_charges). */
int tebd_get_charges(tebd_handle h, int k, int* q);

/* Number of local updates (three-site gates) applied since init, and the
 * number of CUDA kernels this handle has launched since create.
 * Infrastructure: the paper has no counterpart. */
int tebd_counters(tebd_handle h, long long* gate_updates, long long* kernel_launches);

/* Kernel classes timed when the option "profile" is 1. */
enum {
  TEBD_PROF_CONTRACT = 0, /* theta~ = B B B, gate, rebuild of B (complex GEMMs) */
  TEBD_PROF_GRAM = 1,     /* Gram matrices theta' theta'^+ */
  TEBD_PROF_TRIDIAG = 2,  /* Householder reduction of the Gram to tridiagonal form */
  TEBD_PROF_BISECT = 3,   /* eigenvalues by bisection */
  TEBD_PROF_EIGVEC = 4,   /* inverse iteration, orthonormalisation, back-transformation */
  TEBD_PROF_PROJECT = 5,  /* Y = U^+ theta' (singular values and right vectors) */
  TEBD_PROF_TRUNCATE = 6, /* sort, truncation rule, row gathers */
  TEBD_PROF_MEASURE = 7,  /* densities and currents */
  TEBD_PROF_NCLASS = 8
};

/* Infrastructure (no counterpart in the paper).  Totals since the option
 * "profile" was last set to 1: device time in ms (CUDA
 * events on the handle's stream around each group of launches), kernel launches,
 * and algorithmic work (real FP64 flops for classes 0-5, with the Hermitian
 * Gram counted at half and the tridiagonal reduction at 16/3 m^3; bytes of the
 * site tensors read once for class 7).  Any output pointer may be NULL. */
int tebd_profile(tebd_handle h, int cls, double* ms, long long* launches, double* work);

/* Release everything the handle owns.  NULL is accepted.  Infrastructure. */
void tebd_destroy(tebd_handle h);

/* Graph-mode counters (option "graph"): accepted replays, replays undone and run the
 * ordinary way, and the kernel launches one replay holds (0 while no graph is cached).
 * Any pointer may be NULL.  Infrastructure (no counterpart in the paper). */
int tebd_graph_stats(tebd_handle h, long long* replays, long long* fallbacks, long long* launches_per_replay);

/* Static description of a status code.  Infrastructure. */
const char* tebd_strerror(int status);

/* Host-only helper (no GPU needed): the FP64 gate exp(-i h_j tau) of triple
 * j (1-based, 1 <= j <= L-2) as a d^3 x d^3 row-major complex matrix with
 * basis index s1*d^2 + s2*d + s3, written interleaved into out[2*d^6].
 * h_j holds the NNN hop of the triple with weight 1, each NN hop (k,k+1)
 * inside it divided by the number of triples containing that bond, and each
 * on-site term U/2 n(n-1) + K/2 (k-j_c)^2 n divided by the number of triples
 * containing site k, so that sum_j h_j equals eq. (1).  The exponential uses
 * the library's own Hermitian Jacobi eigen-solver. */
int tebd_gate_host(int L, int n_max, double U, double J, double J_NNN, double K, double j_c,
                   int j, double tau, double* out);

/* tebd_gate_host with an explicit sweep limit (max_sweeps >= 1) for the host
 * Jacobi eigen-solver.  The gate built from the sweeps done is written to out
 * either way; TEBD_ERR_NOT_CONVERGED if the off-diagonal weight did not fall
 * below 1e-32 of the Frobenius norm within max_sweeps.  Host only. */
int tebd_gate_host_sweeps(int L, int n_max, double U, double J, double J_NNN, double K, double j_c,
                          int j, double tau, int max_sweeps, double* out);

/* Host-only helper (no GPU needed): the FP64 gate exp(-i h_k tau) of super bond k
 * (1-based, 1 <= k <= L_e - 1, L_e = ceil(L / 2)) of the super-site scheme
 * (tebd_create_supersite) as a d^4 x d^4 row-major complex matrix, d = n_max + 1,
 * over the physical sites (2k-1, 2k, 2k+1, 2k+2) with the last fastest, written
 * interleaved into out[2 d^8]; 1 <= n_max <= 4.  Exponentiated per block of fixed
 * boson number with the library's Hermitian Jacobi eigen-solver. */
int tebd_gate_host_supersite(int L, int n_max, double U, double J, double J_NNN, double K, double j_c,
                             int k, double tau, double* out);

/* The complex contraction used by the local update of Sec. II B (theta, gate,
 * rebuild), exposed for direct use and testing: C = alpha * A * op(B) on device buffers (interleaved complex doubles,
 * row-major with leading dimensions in complex elements), A: M x K, op(B): K x N
 * with opB = 0 (B stored K x N) or 1 (B^+, B stored N x K), C: M x N.
 * precision 0: FP64 on the CUDA cores; 1: split 3xTF32 on the tcgen05 tensor
 * cores with FP32 accumulation (relative error ~5e-7 of |A||B|); 2: FP64-accurate
 * exact-digit products on the bf16 tensor cores (the mixed path's Gram and
 * projection engine: eight 7-bit digits per row-scaled real, exact integer
 * accumulation, one final rounding; error below 2^-53 max|A_i.| max|B_.j| K).
 * Precision 2 allocates and frees its digit workspace stream-ordered on
 * cuda_stream.  Enqueued on cuda_stream (NULL = legacy default stream), not
 * synchronised.  Sizes >= 1, leading dimensions >= the row lengths; otherwise
 * TEBD_ERR_ARG. */
int tebd_zgemm(int precision, int opB, int M, int N, int K, double alpha, const double* A, long long lda,
               const double* B, long long ldb, double* C, long long ldc, void* cuda_stream);

/* Allocation-free nearest-neighbour correlator of one bond.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory when they need the value (a fixed device-memory budget, a
 * framework allocator that must own all device memory, or a latency-critical
 * loop where cudaMalloc would synchronise the device).  It computes
 *   C = <b+_j b_{j+1}> = sum conj(theta[a,s,t,b]) (b+ (x) b) theta[a,s',t',b],
 *   theta = lam_left (.) B_left B_right,
 * the same quantity tebd_measure turns into current_j = 2 J Im C.
 * Inputs (device, caller-owned): B_left [chi_l][d][chi_m] and B_right
 * [chi_m][d][chi_r] as interleaved complex doubles, lam_left [chi_l] doubles.
 * Output (device, caller-owned): C_out[0] = Re C, C_out[1] = Im C.
 * Work is enqueued on cuda_stream (NULL = legacy default stream); the call
 * does not synchronise.  Limits: chi_l, chi_m, chi_r <= 64 and 2 <= d <= 8;
 * larger sizes return TEBD_ERR_TOO_LARGE (with a message on stderr) and
 * launch nothing.
 * Memory: no cudaMalloc, cudaFree or other allocation.  Scratch is a fixed
 * file-scope device array of 1,179,648 bytes, held by every GPU that loads the
 * library until the process exits.  Every call looks up that array's device
 * address (cudaGetSymbolAddress) in the context current on the calling
 * thread, so the address stays right after cudaDeviceReset or under another
 * context; the first call in a context loads the library's device code there,
 * so make it before any stream capture.  All calls on a device share the
 * array, so calls that overlap on the GPU (different streams, or threads
 * without ordering) race and give wrong results; serialise them.
 * Errors: a CUDA error already pending when the call starts (left by other
 * work) is reported as TEBD_ERR_CUDA without clearing it, and nothing is
 * launched; otherwise TEBD_ERR_CUDA reports a failure of this call's own
 * launches. */
int tebd_bond_correlator_noalloc(const double* B_left, const double* lam_left, const double* B_right,
                                 int chi_l, int chi_m, int chi_r, int d, double* C_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* PTEBD_H */
