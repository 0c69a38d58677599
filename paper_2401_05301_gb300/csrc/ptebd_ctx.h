// The handle of the C ABI (struct tebd_ctx) and the host helpers shared by the
// translation units that orchestrate a local update (api.cu: dense tensors;
// u1.cu: the particle-number-blocked form).
#pragma once

#include "ptebd.h"
#include "ptebd_internal.h"

#include <cmath>
#include <cstdio>
#include <utility>
#include <vector>

struct tebd_ctx;

namespace ptebd {

constexpr int MAX_SLOTS = 24;

// Workspace of one local update in flight (dense form).
struct Slot {
  double2 *X, *Th, *Cb, *H, *V1h, *tau, *part, *p, *U;
  double *d, *e, *evals, *Z, *Z2, *S, *work, *s_sorted, *scal;  // scal: [0] trace [1] norm [2] w
  int *perm, *chi;
  double2* pan;  // panel arrays of the blocked tridiagonal reduction
  void* oz;  // digit planes of the mixed path's Gram and projection products (null in FP64)
};

struct Triple {
  tebd_ctx* h;  // the simulation this triple belongs to
  int i;        // 0-based first site
  int slot;
  int chl, c1, c2, chr;
  int m1, n1, K1, chi1, m2, n2, K2, chi2;
  double norm1, norm2, w1, w2;
  long long call;  // randomized truncation: index of cut 1's test matrix (cut 2: call + 1)
  size_t gw1, gw2;  // graph capture: where the two cuts' discarded weights are recorded
};

struct U1Work;  // workspace of the blocked form (u1.cu)

}  // namespace ptebd

struct tebd_ctx {
  int L = 0, n_max = 0, d = 0, D = 0, chi_max = 0;
  // super sites (tebd_create_supersite): the MPS runs on L = L_eff super sites of local
  // dimension d = (n_max + 1)^2 with two-site gates of dimension D = d^2; L_phys physical sites
  bool ss = false;
  int L_phys = 0;
  double U = 0, J = 0, Jnnn = 0, K = 0, jc = 0, dt = 0;
  double w_cut = 0.0, eps_rel = 1e-12;
  int precision = 0, max_slots = 0;
  int order = 2;  // Trotter order: 2 or 4 (gate table and layer schedule follow it)
  int jacobi_sweeps = 60;  // sweep limit of the host gate builder's Jacobi eigen-solver
  long long wait_clocks = 2000000000LL;  // limit of each grid-barrier wait in the reduction (~1 s)
  int panel_blocks = 0;  // blocks per SM of the reduction's cooperative grid (0 = automatic)
  cudaStream_t stream = nullptr;
  int device = 0;
  int sticky = TEBD_OK;
  bool have_state = false;
  std::vector<int> cap, chi;
  std::vector<double2*> B;
  std::vector<double*> lam;
  double2* G = nullptr;
  size_t G_bytes = 0;
  double2** dB = nullptr;
  double** dlam = nullptr;
  int* d_status = nullptr;
  int* d_occ = nullptr;
  unsigned int* d_bar = nullptr;  // grid-barrier state of the persistent reduction
  std::vector<ptebd::Slot> slots;
  long long capmax = 0, mmax = 0, n1max = 0, kcap = 0;
  double* h_pinned = nullptr;
  size_t h_pinned_n = 0;
  double2 *mP = nullptr, *mQ = nullptr, *mX = nullptr, *mY = nullptr, *mC = nullptr;
  double* mN = nullptr;
  double w_total = 0.0;
  long long steps = 0, gate_updates = 0, launches = 0;
  std::vector<void*> allocs;
  size_t alloc_bytes = 0;  // device bytes of allocs
  // particle-number (U(1)) blocked form: option "u1"; q[k] = boson count left of
  // bond k for each Schmidt index, non-decreasing (each charge one contiguous run)
  bool u1 = false;
  bool have_charges = false;
  std::vector<std::vector<int>> q;
  double2* Gblk = nullptr;  // gates restricted to each total-occupation block (u1.cu layout)
  size_t Gblk_n = 0;        // complex elements of Gblk
  ptebd::U1Work* u1w = nullptr;
  // randomized range finder for the truncated SVDs (option "randomized", dense form)
  bool randomized = false;
  int oversample = 10, power_iters = 2;
  tebd_test_matrix_fn omega_fn = nullptr;
  void* omega_ctx = nullptr;
  long long rcall = 0;  // decompositions so far (the test-matrix call index)
  // optional per-class timing (CUDA events on the handle's stream)
  bool prof = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_pending[TEBD_PROF_NCLASS];
  std::vector<int> prof_pending_cls;
  double prof_ms[TEBD_PROF_NCLASS] = {};
  long long prof_launches[TEBD_PROF_NCLASS] = {};
  double prof_work[TEBD_PROF_NCLASS] = {};
  std::vector<cudaEvent_t> event_pool;
  // CUDA-graph replay of whole steps (option "graph", dense three-site form, every bond
  // at capacity): while a step is captured, every decision the host would read back
  // (eigenvector count, chi', norms, status) is fixed to its saturated value and
  // checked on the device instead; a replay whose checks fail is undone from the
  // backup the graph takes first, and the step is run again the ordinary way.
  bool graph = false;
  bool capturing = false;       // the driving handle is being captured
  long long generation = 0;     // bumped by every host change of the state or options
  int* d_gflag = nullptr;       // device: failed checks of the replay (0 = accepted)
  double* d_gw = nullptr;       // device: discarded weights of the captured truncations
  size_t gw_cap = 0, gw_n = 0;
  double* h_gw = nullptr;       // pinned copy of [flag, weights]
  std::vector<std::pair<tebd_ctx*, std::pair<size_t, size_t>>> gw_map;  // (handle, w1, w2 index) per update
  std::vector<std::pair<tebd_ctx*, int>> gcount;  // gate updates per handle per replay
  std::vector<tebd_ctx*> gkey;   // the handles the cached graph steps
  std::vector<long long> ggen;   // their generations at capture
  cudaGraphExec_t gexec = nullptr;
  long long glaunches = 0;       // kernel launches in one replay
  double2* bkB = nullptr;        // backup of the state (B_k then lambda_k, packed by capacity)
  size_t bk_bytes = 0;
  long long graph_replays = 0, graph_fallbacks = 0;
  cudaStream_t own_stream = nullptr;  // created for graph mode when the handle had the legacy stream
  bool graph_broken = false;  // a capture failed: no graph for this handle until "graph" is set again
  int graph_test_fallback = 0;  // diagnostic: undo this many accepted replays as if a check had failed
};

namespace ptebd {

inline bool is_fin(double x) { return std::isfinite(x); }

inline cudaEvent_t get_event(tebd_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

// Times the launches issued during its lifetime as one interval of class cls.
struct ProfScope {
  tebd_ctx* c;
  int cls;
  long long l0;
  cudaEvent_t a = nullptr;
  ProfScope(tebd_ctx* c_, int cls_, double work) : c(c_), cls(cls_), l0(c_->launches) {
    if (!c->prof) return;
    c->prof_work[cls] += work;
    a = get_event(c);
    cudaEventRecord(a, c->stream);
  }
  ~ProfScope() {
    if (!c->prof) return;
    cudaEvent_t b = get_event(c);
    cudaEventRecord(b, c->stream);
    c->prof_pending[cls].push_back({a, b});
    c->prof_launches[cls] += c->launches - l0;
  }
};

template <typename T>
T* dalloc(tebd_ctx* c, size_t count) {
  void* p = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  c->allocs.push_back(p);
  c->alloc_bytes += count * sizeof(T);
  return static_cast<T*>(p);
}

void prof_collect(tebd_ctx* c);
int fail_cuda(tebd_ctx* c);
int check_launch(tebd_ctx* c);
int sync(tebd_ctx* c);
int ensure_pinned(tebd_ctx* c, size_t n);

// ---- particle-number (U(1)) blocked form (u1.cu) ---------------------------------
// One batch of independent local updates with every product and decomposition
// taken block by block over the conserved boson number.
int update_chunk_u1(tebd_ctx* c, std::vector<Triple>& ts, int tidx);
// Gates restricted to their total-occupation blocks, from the dense table (host,
// Gall: ngates x D x D); allocates and fills c->Gblk.
int u1_build_gate_blocks(tebd_ctx* c, const std::vector<std::complex<double>>& Gall, size_t ngates);
// Device bytes of the blocked workspace now held; releases it.
size_t u1_workspace_bytes(const tebd_ctx* c);
void u1_release(tebd_ctx* c);
// nslots workspace slots of the blocked form (their arenas grow on first use).
int u1_alloc_slots(tebd_ctx* c, int nslots);
// Correlators <b+_k b_{k+1}> of every bond (out: device, L-1 complex) from the charge
// blocks of the canonical form; needs the handle's charges.
int u1_correlators(tebd_ctx* h, double2* out);
// Dense form: cut 1 (second = false: theta' = lam C into V1^+) or cut 2 (R into B_{i+2}) of
// every triple by the randomized range finder; sets chi, norm and w of the triples.
int rand_cut(tebd_ctx* c, std::vector<Triple>& ts, bool second);

}  // namespace ptebd
