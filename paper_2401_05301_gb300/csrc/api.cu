// C ABI of the three-site TEBD library: handle, device state, and the host
// orchestration of one Trotter layer (all triples with the same start mod 3
// processed as one batch of independent local updates).
#include "ptebd_ctx.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

using namespace ptebd;

namespace {
constexpr int MEAS_CHUNK = GEMM_MAXP;
}  // namespace

namespace ptebd {

// Fold every finished event pair into the per-class totals (call after a sync).
void prof_collect(tebd_ctx* c) {
  for (int k = 0; k < TEBD_PROF_NCLASS; ++k) {
    for (auto& pr : c->prof_pending[k]) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) c->prof_ms[k] += ms;
      c->event_pool.push_back(pr.first);
      c->event_pool.push_back(pr.second);
    }
    c->prof_pending[k].clear();
  }
  cudaGetLastError();
}

int fail_cuda(tebd_ctx* c) {
  c->sticky = TEBD_ERR_CUDA;
  return TEBD_ERR_CUDA;
}

int check_launch(tebd_ctx* c) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    std::fprintf(stderr, "ptebd: CUDA error %s\n", cudaGetErrorString(e));
    return fail_cuda(c);
  }
  return TEBD_OK;
}

int sync(tebd_ctx* c) {
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    std::fprintf(stderr, "ptebd: CUDA error %s\n", cudaGetErrorString(e));
    return fail_cuda(c);
  }
  if (c->prof) prof_collect(c);
  return TEBD_OK;
}

long long ipow_cap(int d, int e, long long cap) {
  long long v = 1;
  for (int i = 0; i < e; ++i) {
    v *= d;
    if (v >= cap) return cap;
  }
  return std::min(v, cap);
}

int ensure_pinned(tebd_ctx* c, size_t n) {
  if (c->h_pinned_n >= n) return TEBD_OK;
  if (c->h_pinned) cudaFreeHost(c->h_pinned);
  c->h_pinned = nullptr;
  c->h_pinned_n = 0;
  if (cudaMallocHost(&c->h_pinned, n * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return TEBD_ERR_OOM;
  }
  c->h_pinned_n = n;
  return TEBD_OK;
}

}  // namespace ptebd

namespace {

// Device bytes of the blocked form beyond the state, as multiples of the dense theta
// (16 chi^2 d^3): per workspace slot the arenas of one saturated local update (the compact
// theta and C, the packed blocks of both cuts and their eigen-solver buffers), and once
// per handle the exact-digit workspace rings (16 products, 64 eigen-solver matrices, each
// sized for the largest block).  Fitted to tebd_device_bytes of the saturated chi = 1024,
// d = 5, L = 64 state after four steps: 19.7 / 25.2 / 37.9 GB with 4 / 8 / 21 slots (the
// per-slot high-water mark is largest with few slots, each of which sees several triples),
// so the estimate is exact at 4 and 8 slots and 14 % high at 21.
constexpr double U1_ARENA_FRACTION = 0.655;
constexpr double U1_RING_FRACTION = 4.5;

int max_triples_per_layer(int L, bool ss = false) {
  const int stride = ss ? 2 : 3, span = ss ? 1 : 2;  // super sites: NN bonds, two layers
  int best = 0;
  for (int r = 0; r < stride; ++r) {
    int n = 0;
    for (int i = r; i + span < L; i += stride) ++n;
    best = std::max(best, n);
  }
  return best;
}

// Local updates per time index: triples (L - 2) or super bonds (L - 1).
int gate_sites(const tebd_ctx* c) { return c->ss ? c->L - 1 : c->L - 2; }

// Device bytes of one workspace slot (one triple in flight) for bond capacity
// capmax, local dimension d and bond cap chi_max.
// Digit workspace of the mixed path: the largest of the Gram H1 (m x m over n1),
// projection Y1 (K x n1 over m) and projection Y2 (K x m over m) products.
double oz_slot_bytes(long long capmax, long long d, long long chi_max, bool two_site = false) {
  const long long mm = capmax * d, n1max = (two_site ? d : d * d) * capmax, kc = std::min<long long>(mm, chi_max);
  return (double)std::max({oz_workspace_bytes((int)mm, (int)mm, (int)n1max, true),
                           oz_workspace_bytes((int)kc, (int)n1max, (int)mm, false),
                           oz_workspace_bytes((int)kc, (int)mm, (int)mm, false),
                           // contractions of precision 2: B_i B_{i+1}, X B_{i+2}, C V1^+, V1^+ V2^+
                           oz_workspace_bytes((int)mm, (int)(d * capmax), (int)capmax, false),
                           oz_workspace_bytes((int)(mm * d), (int)(d * capmax), (int)capmax, false),
                           oz_workspace_bytes((int)mm, (int)kc, (int)n1max, false),
                           oz_workspace_bytes((int)mm, (int)kc, (int)mm, false)});
}

double slot_bytes_for(long long capmax, long long d, long long chi_max, int precision, bool two_site = false) {
  const long long D = two_site ? d * d : d * d * d, mm = capmax * d, n1max = (two_site ? d : d * d) * capmax;
  const long long kc = std::min<long long>(mm, chi_max);
  // two sites: the projection and V^+ rows (Th, V1h) are at most kc x n1
  const double th_v = two_site ? 2.0 * kc * n1max : capmax * D * capmax + capmax * n1max;
  return 16.0 * (capmax * d * d * capmax + capmax * D * capmax + th_v + mm * mm + 3.0 * mm + EIG_PARTS + kc * mm) +
         8.0 * (4.0 * mm + 4 + 7.0 * mm * kc + kc * kc) + 4.0 * (mm + 1) + 16.0 * eig_panel_doubles2((int)mm) +
         (precision >= 1 ? oz_slot_bytes(capmax, d, chi_max, two_site) : 0.0);
}

std::vector<int> bond_caps(int L, int d, int chi_max) {
  std::vector<int> cap(L + 1);
  for (int k = 0; k <= L; ++k) cap[k] = (int)ipow_cap(d, std::min(k, L - k), chi_max);
  return cap;
}

// Time arguments of the gate table: order 2 uses {dt/2, dt}; order 4 (Suzuki's
// composition S2(p dt)^2 S2((1-4p) dt) S2(p dt)^2, p = 1/(4 - 4^(1/3))) uses
// {p dt/2, p dt, (1-4p) dt/2, (1-4p) dt}.
std::vector<double> gate_taus(const tebd_ctx* c) {
  if (c->order == 2) return {0.5 * c->dt, c->dt};
  const double p = 1.0 / (4.0 - std::cbrt(4.0)), q = 1.0 - 4.0 * p;
  return {0.5 * p * c->dt, p * c->dt, 0.5 * q * c->dt, q * c->dt};
}

// Layers of one step as (residue, index into the gate table): the symmetric
// second-order step A(t/2) B(t/2) C(t) B(t/2) A(t/2), once (order 2) or composed
// five times (order 4).  Adjacent half-step layers are never merged.
std::vector<std::pair<int, int>> step_layers(const tebd_ctx* c) {
  std::vector<std::pair<int, int>> out;
  if (c->ss) {  // super sites: odd bonds dt/2, even bonds dt, odd bonds dt/2 (Sec. II B)
    out = {{0, 0}, {1, 1}, {0, 0}};
    return out;
  }
  auto s2 = [&](int half, int full) {
    const std::pair<int, int> l[5] = {{0, half}, {1, half}, {2, full}, {1, half}, {0, half}};
    out.insert(out.end(), l, l + 5);
  };
  if (c->order == 2) {
    s2(0, 1);
  } else {
    s2(0, 1); s2(0, 1); s2(2, 3); s2(0, 1); s2(0, 1);
  }
  return out;
}

// Build every gate of the table on the host (exact exponentiation) and upload it.
int build_gates(tebd_ctx* c) {
  const size_t DD = (size_t)c->D * c->D, L2 = (size_t)gate_sites(c);
  const std::vector<double> taus = gate_taus(c);
  double2* G = dalloc<double2>(c, taus.size() * L2 * DD);
  if (!G) return TEBD_ERR_OOM;
  std::vector<std::complex<double>> Gall(taus.size() * L2 * DD), Gj;
  for (size_t t = 0; t < taus.size(); ++t)
    for (int j = 1; j <= (int)L2; ++j) {
      const bool ok = c->ss ? build_gate_supersite(c->L_phys, c->n_max, c->U, c->J, c->Jnnn, c->K, c->jc, j, taus[t],
                                                   Gj, c->jacobi_sweeps)
                            : build_gate(c->L, c->n_max, c->U, c->J, c->Jnnn, c->K, c->jc, j, taus[t], Gj,
                                         c->jacobi_sweeps);
      if (!ok) return TEBD_ERR_NOT_CONVERGED;
      std::copy(Gj.begin(), Gj.end(), Gall.begin() + (t * L2 + (j - 1)) * DD);
    }
  if (cudaMemcpy(G, Gall.data(), Gall.size() * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    return TEBD_ERR_CUDA;
  }
  if (!c->ss)
    if (int r = u1_build_gate_blocks(c, Gall, taus.size() * L2)) return r;
  if (c->G) {  // replace the previous table
    for (auto it = c->allocs.begin(); it != c->allocs.end(); ++it)
      if (*it == c->G) { c->allocs.erase(it); break; }
    cudaFree(c->G);
    c->alloc_bytes -= c->G_bytes;
  }
  c->G_bytes = taus.size() * L2 * DD * sizeof(double2);
  c->G = G;
  return TEBD_OK;
}

int alloc_workspace(tebd_ctx* c) {
  if (!c->slots.empty()) return TEBD_OK;
  if (c->u1) {  // the blocked form: slots hold only arenas that grow with the blocks
    int want = std::min(max_triples_per_layer(c->L, c->ss), MAX_SLOTS);
    if (c->max_slots > 0) want = std::min(want, c->max_slots);
    if (int r = u1_alloc_slots(c, want)) return r;
    c->slots.assign(want, Slot{});
    return ensure_pinned(c, 64);
  }
  const long long d = c->d;
  long long capmax = 1;
  for (int v : c->cap) capmax = std::max<long long>(capmax, v);
  c->capmax = capmax;
  c->mmax = capmax * d;
  c->n1max = (c->ss ? d : d * d) * capmax;
  c->kcap = std::min<long long>(c->mmax, c->chi_max);
  if (c->mmax > 12288) return TEBD_ERR_ARG;  // the reduction's partial sums are sized for m <= 12288
  const long long D = c->D, mm = c->mmax, kc = c->kcap;
  const double slot_bytes = slot_bytes_for(capmax, d, c->chi_max, c->precision, c->ss);
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  int want = std::min(max_triples_per_layer(c->L, c->ss), MAX_SLOTS);
  if (c->max_slots > 0) want = std::min(want, c->max_slots);
  const int budget = (int)std::max(1.0, std::floor(0.8 * (double)free_b / slot_bytes));
  const int nslots = std::max(1, std::min(want, budget));
  for (int s = 0; s < nslots; ++s) {
    Slot S{};
    S.X = dalloc<double2>(c, capmax * d * d * capmax);
    S.Th = dalloc<double2>(c, c->ss ? kc * c->n1max : capmax * D * capmax);
    S.Cb = dalloc<double2>(c, capmax * D * capmax);
    S.H = dalloc<double2>(c, mm * mm);
    S.V1h = dalloc<double2>(c, (c->ss ? kc : capmax) * c->n1max);
    S.tau = dalloc<double2>(c, mm);
    S.part = dalloc<double2>(c, EIG_PARTS);
    S.p = dalloc<double2>(c, mm);
    S.U = dalloc<double2>(c, kc * mm);
    S.d = dalloc<double>(c, mm);
    S.e = dalloc<double>(c, mm);
    S.evals = dalloc<double>(c, mm);
    S.Z = dalloc<double>(c, mm * kc);
    S.Z2 = dalloc<double>(c, mm * kc);
    S.S = dalloc<double>(c, kc * kc);
    S.work = dalloc<double>(c, 5 * mm * kc);
    S.s_sorted = dalloc<double>(c, mm);
    S.scal = dalloc<double>(c, 4);
    S.perm = dalloc<int>(c, mm);
    S.chi = dalloc<int>(c, 1);
    S.pan = dalloc<double2>(c, eig_panel_doubles2((int)mm));
    if (c->precision >= 1) S.oz = dalloc<uint8_t>(c, (size_t)oz_slot_bytes(capmax, d, c->chi_max, c->ss));
    if ((c->precision >= 1 && !S.oz) || !S.pan || !S.X || !S.Th || !S.Cb || !S.H || !S.V1h || !S.tau || !S.part || !S.p || !S.U || !S.d || !S.e ||
        !S.evals || !S.Z || !S.Z2 || !S.S || !S.work || !S.s_sorted || !S.scal || !S.perm || !S.chi) {
      if (s == 0) return TEBD_ERR_OOM;
      break;
    }
    c->slots.push_back(S);
  }
  if (c->randomized)  // the range finder's row matrices live in per-slot arenas
    if (int r = u1_alloc_slots(c, (int)c->slots.size())) return r;
  return ensure_pinned(c, (size_t)c->slots.size() * (c->kcap + 8) + 64);
}

// The mixed path's digit planes, for workspaces allocated while the handle was FP64.
int ensure_oz(tebd_ctx* c) {
  for (Slot& S : c->slots)
    if (!S.oz && !(S.oz = dalloc<uint8_t>(c, (size_t)oz_slot_bytes(c->capmax, c->d, c->chi_max, c->ss))))
      return TEBD_ERR_OOM;
  return TEBD_OK;
}

// PTEBD_DEBUG=1: synchronise after each stage and print a summary of a buffer
// (finite count, max |x|) to stderr.  Diagnostic only; off by default.
bool debug_on() {
  static int v = -1;
  if (v < 0) {
    const char* e = std::getenv("PTEBD_DEBUG");
    v = (e && e[0] == '1') ? 1 : 0;
  }
  return v == 1;
}

void debug_dump(tebd_ctx* c, const char* label, int t, const void* ptr, size_t n_doubles) {
  if (!debug_on()) return;
  cudaStreamSynchronize(c->stream);
  std::vector<double> h(n_doubles);
  cudaMemcpy(h.data(), ptr, n_doubles * sizeof(double), cudaMemcpyDeviceToHost);
  size_t bad = 0;
  double mx = 0.0;
  for (double x : h) {
    if (!std::isfinite(x)) ++bad; else mx = std::max(mx, std::fabs(x));
  }
  std::fprintf(stderr, "[ptebd] %-10s t%d n=%zu nonfinite=%zu max=%.3e first=", label, t, n_doubles, bad, mx);
  for (size_t i = 0; i < std::min<size_t>(n_doubles, 6); ++i) std::fprintf(stderr, "%.4e ", h[i]);
  std::fprintf(stderr, "\n");
}

const double2* gate_ptr(const tebd_ctx* c, int i, int tidx) {
  return c->G + ((size_t)tidx * gate_sites(c) + i) * (size_t)c->D * c->D;
}

// Eigen-decomposition of the Gram matrices held in the slots of ts (H, m, kmax
// already set): trace, tridiagonal reduction, bisection, host choice of K,
// eigenvectors.  On return the slots' U hold the K leading eigenvectors.
// c drives the batch (stream, status, pinned buffers); each triple's state,
// slot and options belong to its owner T.h (several simulations may share a batch).
int eigen_stage(tebd_ctx* c, std::vector<Triple>& ts, bool second) {
  EigBatch eb{};
  void* oz_ws[EIG_MAXP] = {};
  eb.n = (int)ts.size();
  eb.bar = c->d_bar;
  eb.wait_clocks = c->wait_clocks;
  eb.panel_blocks = c->panel_blocks;
  for (size_t t = 0; t < ts.size(); ++t) {
    const Slot& S = ts[t].h->slots[ts[t].slot];
    EigMat& M = eb.a[t];
    M.H = S.H; M.d = S.d; M.e = S.e; M.tau = S.tau; M.part = S.part; M.p = S.p;
    M.evals = S.evals; M.trace = S.scal; M.Z = S.Z; M.Z2 = S.Z2; M.S = S.S; M.work = S.work; M.U = S.U;
    M.pan = S.pan;
    oz_ws[t] = S.oz;
    M.m = second ? ts[t].m2 : ts[t].m1;
    const int n = second ? ts[t].n2 : ts[t].n1;
    // at most min(m, n) singular values are non-zero: noise eigenvalues of a
    // rank-deficient Gram matrix must never widen the bond beyond that
    M.kmax = (int)std::min<long long>(std::min(M.m, n), ts[t].h->chi_max);
    M.K = 0;
  }
  {
    double w = 0.0;
    for (int t = 0; t < eb.n; ++t) w += 16.0 / 3.0 * std::pow((double)eb.a[t].m, 3);
    ProfScope ps(c, TEBD_PROF_TRIDIAG, w);
    c->launches += eig_trace(eb, c->stream);
    const int nl = eig_tridiagonalize(eb, c->precision >= 1, oz_ws, c->d_status, c->stream);
    if (nl < 0) {
      cudaGetLastError();
      std::fprintf(stderr, "ptebd: cooperative launch of the tridiagonal reduction refused\n");
      return fail_cuda(c);
    }
    c->launches += nl;
  }
  {
    ProfScope ps(c, TEBD_PROF_BISECT, 0.0);
    c->launches += eig_bisect(eb, c->stream);
  }
  if (int r = check_launch(c)) return r;
  if (c->capturing) {  // all kmax vectors; the device checks that the host would have asked for them
    if (eb.n > GRAPH_MAXT) return TEBD_ERR_STATE;
    GraphEig g{};
    g.n = eb.n;
    g.bar_err = c->d_bar + 2;
    g.flag = c->d_gflag;
    for (int t = 0; t < eb.n; ++t) {
      EigMat& M = eb.a[t];
      g.evals[t] = M.evals;
      g.trace[t] = M.trace;
      g.kmax[t] = M.kmax;
      g.floor_rel[t] = std::max(0.01 * ts[t].h->eps_rel, 1e-15);
      M.K = M.kmax;
      if (second) ts[t].K2 = M.K; else ts[t].K1 = M.K;
    }
    c->launches += launch_graph_check_eig(g, c->stream);
  } else {
  // read back the eigenvalues and the traces
  size_t kmax_all = 1;
  for (int t = 0; t < eb.n; ++t) kmax_all = std::max<size_t>(kmax_all, eb.a[t].kmax);
  const size_t stride = kmax_all + 1;
  if (int r = ensure_pinned(c, ts.size() * stride + 8)) return r;
  for (size_t t = 0; t < ts.size(); ++t) {
    const EigMat& M = eb.a[t];
    cudaMemcpyAsync(c->h_pinned + t * stride, M.evals, sizeof(double) * M.kmax, cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(c->h_pinned + t * stride + kmax_all, M.trace, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  }
  unsigned int* h_bar = reinterpret_cast<unsigned int*>(c->h_pinned + ts.size() * stride);
  cudaMemcpyAsync(h_bar, c->d_bar + 2, sizeof(unsigned int), cudaMemcpyDeviceToHost, c->stream);
  if (int r = sync(c)) return r;
  if (*h_bar != 0) {  // a grid barrier of the reduction timed out: results are invalid
    c->sticky = TEBD_ERR_TIMEOUT;
    return TEBD_ERR_TIMEOUT;
  }
  for (size_t t = 0; t < ts.size(); ++t) {
    EigMat& M = eb.a[t];
    const double* ev = c->h_pinned + t * stride;
    const double trace = c->h_pinned[t * stride + kmax_all];
    if (!is_fin(trace) || !(trace > 0.0)) {
      c->sticky = TEBD_ERR_NONFINITE;
      return TEBD_ERR_NONFINITE;
    }
    // eigenvectors for every eigenvalue that could pass the eps_rel floor (with a
    // 100x margin for the Gram's rounding), at least one.  Below p ~ 1e-15 the
    // Gram matrix's rounding (~eps_mach * trace) hides the singular values, so
    // no vector is computed there whatever eps_rel says.
    const double floor_v = std::max(0.01 * ts[t].h->eps_rel, 1e-15) * trace;
    int K = 0;
    while (K < M.kmax && ev[K] > floor_v) ++K;
    M.K = std::max(1, K);
    if (second) ts[t].K2 = M.K; else ts[t].K1 = M.K;
  }
  }
  for (size_t t = 0; t < ts.size() && !c->capturing; ++t) {
    const EigMat& M = eb.a[t];
    debug_dump(c, "d", ts[t].i, M.d, M.m);
    debug_dump(c, "e", ts[t].i, M.e, M.m);
    debug_dump(c, "evals", ts[t].i, M.evals, M.kmax);
  }
  {
    double w = 0.0;
    for (int t = 0; t < eb.n; ++t) {
      const double m = eb.a[t].m, K = eb.a[t].K;
      w += 8.0 * m * m * K + 12.0 * m * K * K;
    }
    ProfScope ps(c, TEBD_PROF_EIGVEC, w);
    c->launches += eig_vectors(eb, c->precision >= 1, oz_ws, c->d_status, c->stream);
  }
  for (size_t t = 0; t < ts.size() && !c->capturing; ++t) {
    const EigMat& M = eb.a[t];
    debug_dump(c, "Z", ts[t].i, M.Z, (size_t)M.m * M.K);
    debug_dump(c, "Z2", ts[t].i, M.Z2, (size_t)M.m * M.K);
    debug_dump(c, "U", ts[t].i, M.U, 2ull * M.m * M.K);
    if (debug_on()) std::fprintf(stderr, "[ptebd] K=%d m=%d kmax=%d\n", M.K, M.m, M.kmax);
  }
  return check_launch(c);
}

int truncate_stage(tebd_ctx* c, std::vector<Triple>& ts, bool second) {
  TruncBatch tb{};
  tb.n = (int)ts.size();
  for (size_t t = 0; t < ts.size(); ++t) {
    const tebd_ctx* o = ts[t].h;
    const Slot& S = o->slots[ts[t].slot];
    TruncArgs& A = tb.a[t];
    A.Y = S.Th;
    A.K = second ? ts[t].K2 : ts[t].K1;
    A.n = second ? ts[t].n2 : ts[t].n1;
    A.trace = S.scal;
    A.s_sorted = S.s_sorted;
    A.perm = S.perm;
    A.lam_out = o->lam[ts[t].i + (second ? 2 : 1)];
    A.chi_out = S.chi;
    A.norm_out = S.scal + 1;
    A.w_out = S.scal + 2;
    A.w_total = nullptr;
    A.chi_max = std::min(o->chi_max, o->cap[ts[t].i + (second ? 2 : 1)]);
    A.w_cut = o->w_cut;
    A.eps_rel = o->eps_rel;
    A.status = c->d_status;
  }
  {
    ProfScope ps(c, TEBD_PROF_TRUNCATE, 0.0);
    c->launches += launch_truncate(tb, c->stream);
  }
  // chi_max above is also the bond capacity, so chi' can never overrun lam or B
  if (int r = check_launch(c)) return r;
  if (c->capturing) {  // chi' = the bond's capacity, checked on the device; w recorded for the host
    if (ts.size() > (size_t)GRAPH_MAXT) return TEBD_ERR_STATE;
    GraphTrunc g{};
    g.n = (int)ts.size();
    g.status = c->d_status;
    g.flag = c->d_gflag;
    for (size_t t = 0; t < ts.size(); ++t) {
      const tebd_ctx* o = ts[t].h;
      const Slot& S = o->slots[ts[t].slot];
      const int cap = std::min(o->chi_max, o->cap[ts[t].i + (second ? 2 : 1)]);
      if (c->gw_n >= c->gw_cap) return TEBD_ERR_STATE;
      g.chi[t] = S.chi;
      g.expect[t] = cap;
      g.w[t] = S.scal + 2;
      g.w_out[t] = c->d_gw + c->gw_n;
      if (second) { ts[t].chi2 = cap; ts[t].gw2 = c->gw_n; ts[t].norm2 = 1.0; ts[t].w2 = 0.0; }
      else { ts[t].chi1 = cap; ts[t].gw1 = c->gw_n; ts[t].norm1 = 1.0; ts[t].w1 = 0.0; }
      ++c->gw_n;
    }
    c->launches += launch_graph_check_trunc(g, c->stream);
    return check_launch(c);
  }
  const size_t stride = 4;
  if (int r = ensure_pinned(c, ts.size() * stride + 8)) return r;
  for (size_t t = 0; t < ts.size(); ++t) {
    const Slot& S = ts[t].h->slots[ts[t].slot];
    cudaMemcpyAsync(c->h_pinned + t * stride, S.scal + 1, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(reinterpret_cast<int*>(c->h_pinned + t * stride + 2), S.chi, sizeof(int), cudaMemcpyDeviceToHost,
                    c->stream);
  }
  int* h_status = reinterpret_cast<int*>(c->h_pinned + ts.size() * stride);
  cudaMemcpyAsync(h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (int r = sync(c)) return r;
  if (*h_status != 0) {
    c->sticky = *h_status;
    return *h_status;
  }
  for (size_t t = 0; t < ts.size(); ++t) {
    const double* h = c->h_pinned + t * stride;
    const int chi = *reinterpret_cast<const int*>(h + 2);
    if (chi < 1 || chi > ts[t].h->cap[ts[t].i + (second ? 2 : 1)]) {
      c->sticky = TEBD_ERR_STATE;
      return TEBD_ERR_STATE;
    }
    if (second) { ts[t].norm2 = h[0]; ts[t].w2 = h[1]; ts[t].chi2 = chi; }
    else { ts[t].norm1 = h[0]; ts[t].w1 = h[1]; ts[t].chi1 = chi; }
  }
  return TEBD_OK;
}

// C = alpha A op(B) on the exact-digit engine: A is M x K (row stride lda); b(j, k) =
// B[j * b_rs + k * b_ks], conjugated if b_conj (so op(B) = B with (1, ldb), B^+ with (ldb, 1, conj)).
OzProb oz_plain(const double2* A, long long lda, const double2* B, long long b_rs, long long b_ks, int b_conj, int M,
                int N, int K, double2* C, long long ldc, double alpha, void* ws) {
  OzProb q{};
  q.a = OzOperand{A, lda, 1, nullptr, 1, 0};
  q.b = OzOperand{B, b_rs, b_ks, nullptr, 1, b_conj};
  q.M = M;
  q.N = N;
  q.K = K;
  q.C = C;
  q.ldc = ldc;
  q.alpha = alpha;
  q.row_div = q.col_div = 1;
  q.ws = ws;
  return q;
}

// Mixed path, exact-digit tensor-core products (FP64 accuracy):
// Gram H = (lam X)(lam X)^+ of X (m x n, row-major), rows scaled by lam[r / d].
OzProb oz_gram(const double2* X, int m, int n, const double* lam, int d, double2* H, void* ws) {
  OzProb q{};
  q.a = OzOperand{X, n, 1, nullptr, 1, 0};
  q.M = q.N = m;
  q.K = n;
  q.C = H;
  q.ldc = m;
  q.alpha = 1.0;
  q.s_row = q.s_col = lam;
  q.row_div = q.col_div = d;
  q.herm = q.gram = 1;
  q.ws = ws;
  return q;
}

// Projection Y = U^+ (lam X): U holds K eigenvectors as rows of length m, X is m x n.
OzProb oz_project(const double2* U, int K, int m, const double* lam, int d, const double2* X, int n, double2* Y,
                  void* ws) {
  OzProb q{};
  q.a = OzOperand{U, m, 1, lam, d, 1};
  q.b = OzOperand{X, 1, n, nullptr, 1, 0};
  q.M = K;
  q.N = n;
  q.K = m;
  q.C = Y;
  q.ldc = n;
  q.alpha = 1.0;
  q.row_div = q.col_div = 1;
  q.ws = ws;
  return q;
}

// One Newton-Schulz polar step on the rows of the kept right singular vectors,
// V <- (3I - V V^+) V / 2.  Rows formed as u_k^+ theta' / s_k carry overlaps of
// order eps s_1 / s_k with the leading rows; the canonical-form observables and
// the next updates assume orthonormal rows, so the overlaps are removed (the
// step squares the error: from ~1e-10 to rounding).  Scratch: the slot's Gram
// buffer (rows x rows) and Th (rows x n).  second: V2 = B_{i+2}, else V1^+.
int reorthonormalise(tebd_ctx* c, std::vector<Triple>& ts, bool second) {
  cudaStream_t s = c->stream;
  const bool mixed = c->precision >= 1;  // exact-digit products (precision 1 and 2)
  Gemm gG(true, OP_N, OP_C), gA(true, OP_N, OP_N);
  std::vector<OzProb> oG, oA;
  std::vector<PolarArgs> pa;
  double w = 0.0;
  for (auto& T : ts) {
    const Slot& S = T.h->slots[T.slot];
    double2* V = second ? T.h->B[T.i + 2] : S.V1h;
    const int rows = second ? T.chi2 : T.chi1, n = second ? T.n2 : T.n1;
    if (rows <= 0 || n <= 0) continue;
    if (mixed) {
      OzProb g{};
      g.a = OzOperand{V, n, 1, nullptr, 1, 0};
      g.M = g.N = rows; g.K = n; g.C = S.H; g.ldc = rows; g.alpha = 1.0;
      g.row_div = g.col_div = 1; g.gram = g.herm = 1; g.ws = S.oz;
      oG.push_back(g);
      OzProb a{};
      a.a = OzOperand{S.H, rows, 1, nullptr, 1, 0};
      a.b = OzOperand{V, 1, n, nullptr, 1, 0};
      a.M = rows; a.N = n; a.K = rows; a.C = S.Th; a.ldc = n; a.alpha = 1.0;
      a.row_div = a.col_div = 1; a.ws = S.oz;
      oA.push_back(a);
    } else {
      GemmProb& g = gG.add(rows, rows, n, V, n, V, n, S.H, rows);
      g.herm = 1;
      gA.add(rows, n, rows, S.H, rows, V, n, S.Th, n);
    }
    pa.push_back(PolarArgs{S.H, rows});
    w += 12.0 * (double)rows * rows * n;
  }
  ProfScope ps(c, TEBD_PROF_PROJECT, w);
  c->launches += mixed ? oz_gemm_launch(oG, c->d_status, s) : gG.launch(s);
  c->launches += launch_polar_form(pa.data(), (int)pa.size(), s);
  c->launches += mixed ? oz_gemm_launch(oA, c->d_status, s) : gA.launch(s);
  for (auto& T : ts) {
    const Slot& S = T.h->slots[T.slot];
    double2* V = second ? T.h->B[T.i + 2] : S.V1h;
    const int rows = second ? T.chi2 : T.chi1, n = second ? T.n2 : T.n1;
    if (rows <= 0 || n <= 0) continue;
    if (cudaMemcpyAsync(V, S.Th, sizeof(double2) * rows * n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return fail_cuda(c);
  }
  return check_launch(c);
}

// One batch of independent local updates (disjoint triples, possibly of
// different simulations), driven on c's stream.  c->precision selects the
// contraction path for the whole batch.
int update_chunk(tebd_ctx* c, std::vector<Triple>& ts, int tidx) {
  cudaStream_t s = c->stream;
  // precision 1: contractions as split 3xTF32; 2: contractions as exact-digit products.
  // Both: the SVD's dense products on the exact-digit engine (FP64-accurate).
  const bool tf32 = c->precision == 1, exact = c->precision == 2, mixed = c->precision >= 1;
  if (mixed)
    for (auto& T : ts)
      if (int r = ensure_oz(T.h)) return r;
  const bool two = c->ss;  // super sites: theta~ = B_i B_{i+1}, one cut, B_{i+1} = V^+
  for (auto& T : ts) {
    const tebd_ctx* o = T.h;
    T.chl = o->chi[T.i]; T.c1 = o->chi[T.i + 1]; T.c2 = o->chi[T.i + 2];
    T.chr = two ? T.c2 : o->chi[T.i + 3];
    T.m1 = T.chl * o->d;
    T.n1 = (two ? o->d : o->d * o->d) * T.chr;
  }
  // theta~ = B_i B_{i+1} B_{i+2}; C = G theta~; Gram H1 = (lam C)(lam C)^+
  {
    Gemm g1(true, OP_N, OP_N), g2(true, OP_N, OP_N), g3(true, OP_N, OP_N), g4(true, OP_N, OP_C);
    std::vector<OzProb> oz4;
    for (auto& T : ts) {
      tebd_ctx* o = T.h;
      const int d = o->d, D = o->D;
      const Slot& S = o->slots[T.slot];
      g1.add(T.chl * d, d * T.c2, T.c1, o->B[T.i], T.c1, o->B[T.i + 1], (long long)d * T.c2, S.X, (long long)d * T.c2);
      if (!two)
        g2.add(T.chl * d * d, d * T.chr, T.c2, S.X, T.c2, o->B[T.i + 2], (long long)d * T.chr, S.Th,
               (long long)d * T.chr);
      GemmProb& p3 = g3.add(D, T.chr, D, gate_ptr(o, T.i, tidx), D, two ? S.X : S.Th, T.chr, S.Cb, T.chr);
      p3.batch = T.chl;
      p3.sA = 0;
      p3.sB = p3.sC = (long long)D * T.chr;
      GemmProb& p4 = g4.add(T.m1, T.m1, T.n1, S.Cb, T.n1, S.Cb, T.n1, S.H, T.m1);
      p4.s_row = p4.s_col = o->lam[T.i];
      p4.row_div = p4.col_div = d;
      p4.herm = 1;
      oz4.push_back(oz_gram(S.Cb, T.m1, T.n1, o->lam[T.i], d, S.H, S.oz));
    }
    double wc = 0.0, wg = 0.0;
    for (auto& T : ts) {
      const double d = T.h->d, D = T.h->D;
      wc += 8.0 * ((double)T.chl * d * d * T.c2 * T.c1 + (two ? 0.0 : (double)T.chl * d * d * d * T.chr * T.c2) +
                   D * D * T.chr * T.chl);
      wg += 4.0 * (double)T.m1 * T.m1 * T.n1;
    }
    {
      ProfScope ps(c, TEBD_PROF_CONTRACT, wc);
      if (exact) {  // X = B_i B_{i+1}, then Th = X B_{i+2}; the gate stays on the FP64 GEMM
        std::vector<OzProb> o1, o2;
        for (auto& T : ts) {
          tebd_ctx* o = T.h;
          const int d = o->d;
          const Slot& S = o->slots[T.slot];
          o1.push_back(oz_plain(o->B[T.i], T.c1, o->B[T.i + 1], 1, (long long)d * T.c2, 0, T.chl * d, d * T.c2, T.c1,
                                S.X, (long long)d * T.c2, 1.0, S.oz));
          if (!two)
            o2.push_back(oz_plain(S.X, T.c2, o->B[T.i + 2], 1, (long long)d * T.chr, 0, T.chl * d * d, d * T.chr,
                                  T.c2, S.Th, (long long)d * T.chr, 1.0, S.oz));
        }
        c->launches += oz_gemm_launch(o1, c->d_status, s);
        c->launches += oz_gemm_launch(o2, c->d_status, s);
        c->launches += g3.launch(s);
      } else {
        c->launches += g1.launch(s, tf32, c->d_status);
        c->launches += g2.launch(s, tf32, c->d_status);
        c->launches += g3.launch(s, tf32, c->d_status);
      }
    }
    if (!c->randomized) {  // the randomized cut never forms the Gram matrix of theta'
      ProfScope ps(c, TEBD_PROF_GRAM, wg);
      c->launches += mixed ? oz_gemm_launch(oz4, c->d_status, s) : g4.launch(s);
    }
    if (int r = check_launch(c)) return r;
    for (auto& T : ts) {
      const Slot& S = T.h->slots[T.slot];
      const int d = T.h->d;
      debug_dump(c, "X", T.i, S.X, 2ull * T.chl * d * d * T.c2);
      debug_dump(c, "Theta", T.i, S.Th, 2ull * T.m1 * T.n1);
      debug_dump(c, "C", T.i, S.Cb, 2ull * T.m1 * T.n1);
      debug_dump(c, "H1", T.i, S.H, 2ull * T.m1 * T.m1);
    }
  }
  if (c->randomized) {
    if (int r = rand_cut(c, ts, false)) return r;
  } else {
  if (int r = eigen_stage(c, ts, false)) return r;
  {  // Y1 = U1^+ (lam C)
    Gemm g5(true, OP_CJ, OP_N);
    std::vector<OzProb> oz5;
    for (auto& T : ts) {
      const Slot& S = T.h->slots[T.slot];
      GemmProb& p = g5.add(T.K1, T.n1, T.m1, S.U, T.m1, S.Cb, T.n1, S.Th, T.n1);
      p.s_red = T.h->lam[T.i];
      p.red_div = T.h->d;
      oz5.push_back(oz_project(S.U, T.K1, T.m1, T.h->lam[T.i], T.h->d, S.Cb, T.n1, S.Th, S.oz));
    }
    double w = 0.0;
    for (auto& T : ts) w += 8.0 * (double)T.K1 * T.n1 * T.m1;
    ProfScope ps(c, TEBD_PROF_PROJECT, w);
    c->launches += mixed ? oz_gemm_launch(oz5, c->d_status, s) : g5.launch(s);
  }
  for (auto& T : ts) debug_dump(c, "Y1", T.i, T.h->slots[T.slot].Th, 2ull * T.K1 * T.n1);
  if (int r = truncate_stage(c, ts, false)) return r;
  {
    std::vector<GatherArgs> ga;
    for (auto& T : ts) {
      const Slot& S = T.h->slots[T.slot];
      ga.push_back(GatherArgs{S.Th, S.perm, S.s_sorted, S.V1h, T.chi1, T.n1});
    }
    {
      ProfScope ps(c, TEBD_PROF_TRUNCATE, 0.0);
      c->launches += launch_gather_rows(ga.data(), (int)ga.size(), s);
    }
    if (int r = reorthonormalise(c, ts, false)) return r;
  }
  }
  {
    // B_i = C V1 / ||s||;  Gram H2 = (lam' V1^+)(lam' V1^+)^+ viewed as (chi' d) x (d chr)
    Gemm g6(true, OP_N, OP_C), g7(true, OP_N, OP_C);
    std::vector<OzProb> oz7;
    for (auto& T : ts) {
      tebd_ctx* o = T.h;
      const int d = o->d;
      const Slot& S = o->slots[T.slot];
      T.m2 = T.chi1 * d;
      T.n2 = d * T.chr;
      GemmProb& p6 = g6.add(T.m1, T.chi1, T.n1, S.Cb, T.n1, S.V1h, T.n1, o->B[T.i], T.chi1);
      p6.alpha_re = 1.0 / T.norm1;
      GemmProb& p7 = g7.add(T.m2, T.m2, T.n2, S.V1h, T.n2, S.V1h, T.n2, S.H, T.m2);
      p7.s_row = p7.s_col = o->lam[T.i + 1];
      p7.row_div = p7.col_div = d;
      p7.herm = 1;
      oz7.push_back(oz_gram(S.V1h, T.m2, T.n2, o->lam[T.i + 1], d, S.H, S.oz));
    }
    double wc = 0.0, wg = 0.0;
    for (auto& T : ts) {
      wc += 8.0 * (double)T.m1 * T.chi1 * T.n1;
      if (!two) wg += 4.0 * (double)T.m2 * T.m2 * T.n2;
    }
    {
      ProfScope ps(c, TEBD_PROF_CONTRACT, wc);
      if (exact) {  // B_i = C V1^+ / ||s||
        std::vector<OzProb> o6;
        for (auto& T : ts) {
          const Slot& S = T.h->slots[T.slot];
          o6.push_back(oz_plain(S.Cb, T.n1, S.V1h, T.n1, 1, 1, T.m1, T.chi1, T.n1, T.h->B[T.i], T.chi1,
                                1.0 / T.norm1, S.oz));
        }
        c->launches += oz_gemm_launch(o6, c->d_status, s);
      } else {
        c->launches += g6.launch(s, tf32, c->d_status);
      }
      if (c->capturing)  // B_i / ||s|| with the norm the truncation left on the device
        for (auto& T : ts)
          c->launches += launch_scale_inv(T.h->B[T.i], (long long)T.m1 * T.chi1, T.h->slots[T.slot].scal + 1, s);
    }
    if (!c->randomized && !two) {
      ProfScope ps(c, TEBD_PROF_GRAM, wg);
      c->launches += mixed ? oz_gemm_launch(oz7, c->d_status, s) : g7.launch(s);
    }
    if (int r = check_launch(c)) return r;
  }
  if (two) {  // B_{i+1} = V^+ (chi' x d chr, rows orthonormal)
    for (auto& T : ts) {
      const Slot& S = T.h->slots[T.slot];
      if (cudaMemcpyAsync(T.h->B[T.i + 1], S.V1h, sizeof(double2) * (size_t)T.chi1 * T.n1, cudaMemcpyDeviceToDevice,
                          s) != cudaSuccess)
        return fail_cuda(c);
    }
    for (auto& T : ts) {
      T.h->chi[T.i + 1] = T.chi1;
      T.h->w_total += T.w1;
      T.h->gate_updates += 1;
    }
    return check_launch(c);
  }
  if (c->randomized) {
    if (int r = rand_cut(c, ts, true)) return r;
  } else {
  if (int r = eigen_stage(c, ts, true)) return r;
  {  // Y2 = U2^+ (lam' V1^+)
    Gemm g8(true, OP_CJ, OP_N);
    std::vector<OzProb> oz8;
    for (auto& T : ts) {
      const Slot& S = T.h->slots[T.slot];
      GemmProb& p = g8.add(T.K2, T.n2, T.m2, S.U, T.m2, S.V1h, T.n2, S.Th, T.n2);
      p.s_red = T.h->lam[T.i + 1];
      p.red_div = T.h->d;
      oz8.push_back(oz_project(S.U, T.K2, T.m2, T.h->lam[T.i + 1], T.h->d, S.V1h, T.n2, S.Th, S.oz));
    }
    double w = 0.0;
    for (auto& T : ts) w += 8.0 * (double)T.K2 * T.n2 * T.m2;
    ProfScope ps(c, TEBD_PROF_PROJECT, w);
    c->launches += mixed ? oz_gemm_launch(oz8, c->d_status, s) : g8.launch(s);
  }
  if (int r = truncate_stage(c, ts, true)) return r;
  {
    std::vector<GatherArgs> ga;
    for (auto& T : ts) {
      const Slot& S = T.h->slots[T.slot];
      ga.push_back(GatherArgs{S.Th, S.perm, S.s_sorted, T.h->B[T.i + 2], T.chi2, T.n2});
    }
    {
      ProfScope ps(c, TEBD_PROF_TRUNCATE, 0.0);
      c->launches += launch_gather_rows(ga.data(), (int)ga.size(), s);
    }
    if (int r = reorthonormalise(c, ts, true)) return r;
  }
  }
  {
    // B_{i+1} = V1^+ V2 / ||s2||,  B_{i+2} = V2^+ (gathered above)
    Gemm g9(true, OP_N, OP_C);
    for (auto& T : ts) {
      tebd_ctx* o = T.h;
      const Slot& S = o->slots[T.slot];
      GemmProb& p = g9.add(T.m2, T.chi2, T.n2, S.V1h, T.n2, o->B[T.i + 2], T.n2, o->B[T.i + 1], T.chi2);
      p.alpha_re = 1.0 / T.norm2;
    }
    double w = 0.0;
    for (auto& T : ts) w += 8.0 * (double)T.m2 * T.chi2 * T.n2;
    {
      ProfScope ps(c, TEBD_PROF_CONTRACT, w);
      if (exact) {  // B_{i+1} = V1^+ V2 / ||s2||
        std::vector<OzProb> o9;
        for (auto& T : ts) {
          const Slot& S = T.h->slots[T.slot];
          o9.push_back(oz_plain(S.V1h, T.n2, T.h->B[T.i + 2], T.n2, 1, 1, T.m2, T.chi2, T.n2, T.h->B[T.i + 1],
                                T.chi2, 1.0 / T.norm2, S.oz));
        }
        c->launches += oz_gemm_launch(o9, c->d_status, s);
      } else {
        c->launches += g9.launch(s, tf32, c->d_status);
      }
      if (c->capturing)
        for (auto& T : ts)
          c->launches += launch_scale_inv(T.h->B[T.i + 1], (long long)T.m2 * T.chi2, T.h->slots[T.slot].scal + 1, s);
    }
    if (int r = check_launch(c)) return r;
  }
  for (auto& T : ts) {
    T.h->chi[T.i + 1] = T.chi1;
    T.h->chi[T.i + 2] = T.chi2;
    if (c->capturing) {  // accounted when a replay is accepted
      c->gw_map.push_back({T.h, {T.gw1, T.gw2}});
      continue;
    }
    T.h->w_total += T.w1 + T.w2;
    T.h->gate_updates += 1;
  }
  return TEBD_OK;
}

// One Trotter layer (triples i = residue mod 3, time index tidx) of every
// simulation in hs, as chunks of at most chunk_max triples in which each
// simulation uses at most its own number of workspace slots.  c drives.
int run_layer_multi(tebd_ctx* c, const std::vector<tebd_ctx*>& hs, int residue, int tidx) {
  struct Pending { tebd_ctx* h; int i; };
  std::vector<Pending> rest;
  const int stride = c->ss ? 2 : 3, span = c->ss ? 1 : 2;
  for (tebd_ctx* h : hs)
    for (int i = residue; i + span < h->L; i += stride) rest.push_back({h, i});
  for (tebd_ctx* h : hs)  // a randomized simulation needs the workspace arenas (switched on late)
    if (h->randomized)
      if (int r = u1_alloc_slots(h, (int)h->slots.size())) return r;
  // Each chunk takes, in order, every pending triple whose simulation still has a free
  // workspace slot in this chunk, up to chunk_max triples; the triples of a layer are
  // disjoint, so any grouping gives the same (bitwise) result.
  const int chunk_max = c->u1 ? 64 : CHUNK_MAXP;  // the blocked form has no fixed-size batches
  while (!rest.empty()) {
    std::vector<Triple> ts;
    std::vector<std::pair<tebd_ctx*, int>> used;  // slots taken per simulation in this chunk
    std::vector<Pending> later;
    for (const Pending& p : rest) {
      int* k = nullptr;
      for (auto& u : used)
        if (u.first == p.h) k = &u.second;
      const int taken = k ? *k : 0;
      if ((int)ts.size() >= chunk_max || taken >= (int)p.h->slots.size()) {
        later.push_back(p);
        continue;
      }
      Triple T{};
      T.h = p.h;
      T.i = p.i;
      T.slot = taken;
      T.call = p.h->rcall + 2 * ((p.i - residue) / stride);
      ts.push_back(T);
      if (k) ++*k; else used.push_back({p.h, 1});
    }
    if (int r = c->u1 ? update_chunk_u1(c, ts, tidx) : update_chunk(c, ts, tidx)) return r;
    rest.swap(later);
  }
  for (tebd_ctx* h : hs)
    for (int i = residue; i + span < h->L; i += stride) h->rcall += 2;
  return TEBD_OK;
}

int run_layer(tebd_ctx* c, int residue, int tidx) { return run_layer_multi(c, {c}, residue, tidx); }

// ---- CUDA-graph replay of whole steps --------------------------------------------------
bool saturated(const tebd_ctx* h) {
  for (int k = 0; k <= h->L; ++k)
    if (h->chi[k] != std::min(h->chi_max, h->cap[k])) return false;
  return true;
}

bool graph_eligible(const std::vector<tebd_ctx*>& hs) {
  for (const tebd_ctx* h : hs)
    if (!h->graph || h->graph_broken || h->prof || h->u1 || h->ss || h->randomized || !h->have_state ||
        !saturated(h))
      return false;
  return true;
}

void graph_drop(tebd_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
  c->gkey.clear();
  c->ggen.clear();
}

bool graph_key_matches(const tebd_ctx* c, const std::vector<tebd_ctx*>& hs) {
  if (c->gkey != hs || c->ggen.size() != hs.size()) return false;
  for (size_t i = 0; i < hs.size(); ++i)
    if (c->ggen[i] != hs[i]->generation) return false;
  return true;
}

// Copy the whole state (every B_k and lambda_k at capacity) to the handle's backup, or back.
int state_copy(tebd_ctx* h, bool restore, cudaStream_t s) {
  size_t need = 0;
  for (int k = 0; k < h->L; ++k) need += 16 * (size_t)h->cap[k] * h->d * h->cap[k + 1];
  for (int k = 0; k <= h->L; ++k) need += 8 * (size_t)h->cap[k];
  if (h->bk_bytes < need) {
    if (restore) return TEBD_ERR_STATE;
    h->bkB = dalloc<double2>(h, (need + 15) / 16);
    if (!h->bkB) return TEBD_ERR_OOM;
    h->bk_bytes = need;
  }
  char* base = reinterpret_cast<char*>(h->bkB);
  size_t off = 0;
  for (int k = 0; k < h->L; ++k) {
    const size_t n = 16 * (size_t)h->cap[k] * h->d * h->cap[k + 1];
    if (cudaMemcpyAsync(restore ? (void*)h->B[k] : (void*)(base + off), restore ? (const void*)(base + off) : h->B[k], n,
                        cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return fail_cuda(h);
    off += n;
  }
  for (int k = 0; k <= h->L; ++k) {
    const size_t n = 8 * (size_t)h->cap[k];
    if (cudaMemcpyAsync(restore ? (void*)h->lam[k] : (void*)(base + off), restore ? (const void*)(base + off) : h->lam[k],
                        n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return fail_cuda(h);
    off += n;
  }
  return TEBD_OK;
}

// One step of the simulations hs (driven on c's stream) by replaying a captured graph.
// Returns TEBD_OK if the replay was accepted, 1 if the step must run the ordinary way
// (not eligible, first step of a new set, or a failed check, the state then restored),
// or an error.  A graph is captured on the second consecutive eligible step of the same
// simulations, after an ordinary step has made every lazy allocation.
int graph_step(tebd_ctx* c, const std::vector<tebd_ctx*>& hs, const std::vector<std::pair<int, int>>& layers) {
  if (!graph_eligible(hs) || c->stream == nullptr) {  // capture needs a stream other than the legacy one
    graph_drop(c);
    return 1;
  }
  if (!graph_key_matches(c, hs)) {  // remember the set; capture on its next step
    graph_drop(c);
    c->gkey = hs;
    for (const tebd_ctx* h : hs) c->ggen.push_back(h->generation);
    return 1;
  }
  if (!c->gexec) {
    size_t ncut = 0;
    for (const tebd_ctx* h : hs)
      for (const auto& l : layers) {
        const int stride = 3, span = 2;
        for (int i = l.first; i + span < h->L; i += stride) ncut += 2;
      }
    if (!c->d_gflag && !(c->d_gflag = dalloc<int>(c, 1))) return TEBD_ERR_OOM;
    if (c->gw_cap < ncut) {
      c->d_gw = dalloc<double>(c, ncut);
      if (!c->d_gw) return TEBD_ERR_OOM;
      if (c->h_gw) cudaFreeHost(c->h_gw);
      c->h_gw = nullptr;
      if (cudaMallocHost(&c->h_gw, sizeof(double) * (ncut + 2)) != cudaSuccess) {
        cudaGetLastError();
        return TEBD_ERR_OOM;
      }
      c->gw_cap = ncut;
    }
    for (tebd_ctx* h : hs)  // the backup buffers, allocated outside the capture
      if (h->bk_bytes == 0 && state_copy(h, false, c->stream) != TEBD_OK) return TEBD_ERR_OOM;
    if (int r = sync(c)) return r;
    c->gw_n = 0;
    c->gw_map.clear();
    const long long l0 = c->launches;
    std::vector<int> sticky0;
    for (const tebd_ctx* h : hs) sticky0.push_back(h->sticky);
    if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      graph_drop(c);
      return 1;
    }
    c->capturing = true;
    int r = cudaMemsetAsync(c->d_gflag, 0, sizeof(int), c->stream) == cudaSuccess ? TEBD_OK : TEBD_ERR_CUDA;
    for (tebd_ctx* h : hs)
      if (r == TEBD_OK) r = state_copy(h, false, c->stream);
    for (size_t l = 0; l < layers.size() && r == TEBD_OK; ++l) r = run_layer_multi(c, hs, layers[l].first, layers[l].second);
    c->capturing = false;
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(c->stream, &g);
    if (r == TEBD_OK && ec == cudaSuccess && g && cudaGraphInstantiate(&c->gexec, g, 0) == cudaSuccess) {
      c->glaunches = c->launches - l0;
    } else {
      cudaGetLastError();
      c->gexec = nullptr;
    }
    if (g) cudaGraphDestroy(g);
    c->launches = l0;
    for (size_t i = 0; i < hs.size(); ++i) hs[i]->sticky = sticky0[i];  // nothing ran during the capture
    if (!c->gexec) {
      graph_drop(c);
      c->graph_broken = true;
      return 1;
    }
  }
  if (cudaGraphLaunch(c->gexec, c->stream) != cudaSuccess) return fail_cuda(c);
  int* h_flag = reinterpret_cast<int*>(c->h_gw);
  cudaMemcpyAsync(h_flag, c->d_gflag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  cudaMemcpyAsync(c->h_gw + 2, c->d_gw, sizeof(double) * c->gw_n, cudaMemcpyDeviceToHost, c->stream);
  if (int r = sync(c)) return r;
  if (c->graph_test_fallback > 0 && *h_flag == 0) {
    --c->graph_test_fallback;
    *h_flag = 32;
  }
  if (*h_flag == 0) {
    const double* w = c->h_gw + 2;
    for (const auto& e : c->gw_map) {
      e.first->w_total += w[e.second.first] + w[e.second.second];
      e.first->gate_updates += 1;
    }
    c->launches += c->glaunches;
    ++c->graph_replays;
    return TEBD_OK;
  }
  for (tebd_ctx* h : hs)
    if (int r = state_copy(h, true, c->stream)) return r;
  if (int r = sync(c)) return r;
  ++c->graph_fallbacks;
  graph_drop(c);
  return 1;
}

int ensure_measure_ws(tebd_ctx* c) {
  if (!c->mN) {  // super sites: two physical densities per site, 2L - 1 physical bonds
    c->mC = dalloc<double2>(c, c->ss ? 2 * c->L : c->L);
    c->mN = dalloc<double>(c, c->ss ? 2 * c->L : c->L);
    if (!c->mC || !c->mN) return TEBD_ERR_OOM;
  }
  if (c->u1 && c->have_charges) return TEBD_OK;  // the blocked correlators use their own arena
  if (!c->mP) {
    const long long capmax = std::max<long long>(1, *std::max_element(c->cap.begin(), c->cap.end()));
    const long long big = capmax * c->d * capmax;
    c->mP = dalloc<double2>(c, MEAS_CHUNK * big);
    c->mQ = dalloc<double2>(c, MEAS_CHUNK * big);
    c->mX = dalloc<double2>(c, MEAS_CHUNK * capmax * capmax);
    c->mY = dalloc<double2>(c, MEAS_CHUNK * capmax * capmax);
    if (!c->mP || !c->mQ || !c->mX || !c->mY) return TEBD_ERR_OOM;
  }
  return TEBD_OK;
}

#define CHECK_HANDLE(h)                         \
  do {                                          \
    if (!(h)) return TEBD_ERR_ARG;              \
    if ((h)->sticky != TEBD_OK) return (h)->sticky; \
  } while (0)

}  // namespace

extern "C" {

const char* tebd_strerror(int status) {
  switch (status) {
    case TEBD_OK: return "ok";
    case TEBD_ERR_ARG: return "invalid argument";
    case TEBD_ERR_OOM: return "device allocation failed";
    case TEBD_ERR_CUDA: return "CUDA error";
    case TEBD_ERR_STATE: return "call out of order";
    case TEBD_ERR_NOT_CONVERGED: return "iteration limit reached";
    case TEBD_ERR_TIMEOUT: return "device wait timed out";
    case TEBD_ERR_NONFINITE: return "non-finite singular values";
    case TEBD_ERR_TOO_LARGE: return "size exceeds the fixed scratch capacity";
    default: return "unknown status";
  }
}

int tebd_zgemm(int precision, int opB, int M, int N, int K, double alpha, const double* A, long long lda,
               const double* B, long long ldb, double* C, long long ldc, void* cuda_stream) {
  if (precision < 0 || precision > 2 || (opB != 0 && opB != 1)) return TEBD_ERR_ARG;
  if (M < 1 || N < 1 || K < 1 || !A || !B || !C || !is_fin(alpha)) return TEBD_ERR_ARG;
  if (lda < K || ldc < N || ldb < (opB ? K : N)) return TEBD_ERR_ARG;
  if (precision == 2) {
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    OzProb q{};
    q.a = OzOperand{reinterpret_cast<const double2*>(A), lda, 1, nullptr, 1, 0};
    q.b = opB ? OzOperand{reinterpret_cast<const double2*>(B), ldb, 1, nullptr, 1, 1}
              : OzOperand{reinterpret_cast<const double2*>(B), 1, ldb, nullptr, 1, 0};
    q.M = M;
    q.N = N;
    q.K = K;
    q.C = reinterpret_cast<double2*>(C);
    q.ldc = ldc;
    q.alpha = alpha;
    q.row_div = q.col_div = 1;
    if (cudaMallocAsync(&q.ws, oz_workspace_bytes(M, N, K, false), st) != cudaSuccess) {
      cudaGetLastError();
      return TEBD_ERR_OOM;
    }
    try {
      oz_gemm_launch({q}, nullptr, st);
    } catch (...) {
      cudaFreeAsync(q.ws, st);
      return TEBD_ERR_OOM;
    }
    cudaFreeAsync(q.ws, st);
    return cudaGetLastError() == cudaSuccess ? TEBD_OK : TEBD_ERR_CUDA;
  }
  try {
    Gemm g(true, OP_N, opB ? OP_C : OP_N);
    GemmProb& p = g.add(M, N, K, A, lda, B, ldb, C, ldc);
    p.alpha_re = alpha;
    g.launch(static_cast<cudaStream_t>(cuda_stream), precision == 1, nullptr);
  } catch (...) {
    return TEBD_ERR_OOM;
  }
  return cudaGetLastError() == cudaSuccess ? TEBD_OK : TEBD_ERR_CUDA;
}

int tebd_gate_host(int L, int n_max, double U, double J, double J_NNN, double K, double j_c, int j, double tau,
                   double* out) {
  if (L < 3 || n_max < 1 || n_max > 7 || j < 1 || j > L - 2 || !out) return TEBD_ERR_ARG;
  if (!is_fin(U) || !is_fin(J) || !is_fin(J_NNN) || !is_fin(K) || !is_fin(j_c) || !is_fin(tau)) return TEBD_ERR_ARG;
  try {
    std::vector<std::complex<double>> G;
    if (!build_gate(L, n_max, U, J, J_NNN, K, j_c, j, tau, G)) return TEBD_ERR_NOT_CONVERGED;
    std::memcpy(out, G.data(), G.size() * sizeof(std::complex<double>));
  } catch (...) {
    return TEBD_ERR_OOM;
  }
  return TEBD_OK;
}

int tebd_gate_host_supersite(int L, int n_max, double U, double J, double J_NNN, double K, double j_c, int k,
                             double tau, double* out) {
  const int L_e = (L + L % 2) / 2;
  if (L < 3 || n_max < 1 || n_max > 4 || k < 1 || k > L_e - 1 || !out) return TEBD_ERR_ARG;
  if (!is_fin(U) || !is_fin(J) || !is_fin(J_NNN) || !is_fin(K) || !is_fin(j_c) || !is_fin(tau)) return TEBD_ERR_ARG;
  try {
    std::vector<std::complex<double>> G;
    const bool ok = build_gate_supersite(L, n_max, U, J, J_NNN, K, j_c, k, tau, G, 60);
    std::memcpy(out, G.data(), G.size() * sizeof(std::complex<double>));
    if (!ok) return TEBD_ERR_NOT_CONVERGED;
  } catch (...) {
    return TEBD_ERR_OOM;
  }
  return TEBD_OK;
}

int tebd_gate_host_sweeps(int L, int n_max, double U, double J, double J_NNN, double K, double j_c, int j,
                          double tau, int max_sweeps, double* out) {
  if (L < 3 || n_max < 1 || n_max > 7 || j < 1 || j > L - 2 || !out || max_sweeps < 1) return TEBD_ERR_ARG;
  if (!is_fin(U) || !is_fin(J) || !is_fin(J_NNN) || !is_fin(K) || !is_fin(j_c) || !is_fin(tau)) return TEBD_ERR_ARG;
  try {
    std::vector<std::complex<double>> G;
    const bool ok = build_gate(L, n_max, U, J, J_NNN, K, j_c, j, tau, G, max_sweeps);
    std::memcpy(out, G.data(), G.size() * sizeof(std::complex<double>));
    if (!ok) return TEBD_ERR_NOT_CONVERGED;
  } catch (...) {
    return TEBD_ERR_OOM;
  }
  return TEBD_OK;
}

}  // extern "C"

namespace {

// L is the chain the MPS runs on (super sites when ss); L_phys the physical length.
int create_impl(int L, int L_phys, bool ss, int n_max, int chi_max, double U, double J, double J_NNN, double K,
                double j_c, double dt, tebd_handle* out) {
  if (!out) return TEBD_ERR_ARG;
  *out = nullptr;
  if (!is_fin(U) || !is_fin(J) || !is_fin(J_NNN) || !is_fin(K) || !is_fin(j_c) || !is_fin(dt) || !(dt > 0))
    return TEBD_ERR_ARG;
  tebd_ctx* c = nullptr;
  try {
    c = new tebd_ctx();
  } catch (...) {
    return TEBD_ERR_OOM;
  }
  c->L = L; c->n_max = n_max; c->chi_max = chi_max;
  c->ss = ss;
  c->L_phys = L_phys;
  c->d = ss ? (n_max + 1) * (n_max + 1) : n_max + 1;
  c->D = ss ? c->d * c->d : c->d * c->d * c->d;
  c->U = U; c->J = J; c->Jnnn = J_NNN; c->K = K; c->jc = j_c; c->dt = dt;
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return TEBD_ERR_CUDA;
  }
  try {
    c->cap = bond_caps(L, c->d, chi_max);
    c->chi.assign(L + 1, 1);
    c->B.resize(L);
    c->lam.resize(L + 1);
    for (int k = 0; k < L; ++k) {
      c->B[k] = dalloc<double2>(c, (size_t)c->cap[k] * c->d * c->cap[k + 1]);
      if (!c->B[k]) throw std::bad_alloc();
    }
    for (int k = 0; k <= L; ++k) {
      c->lam[k] = dalloc<double>(c, c->cap[k]);
      if (!c->lam[k]) throw std::bad_alloc();
    }
    c->dB = dalloc<double2*>(c, L);
    c->dlam = dalloc<double*>(c, L + 1);
    c->d_status = dalloc<int>(c, 1);
    c->d_occ = dalloc<int>(c, L);
    c->d_bar = dalloc<unsigned int>(c, 4);
    if (int r = build_gates(c)) {
      tebd_destroy(c);
      return r;
    }
    if (!c->dB || !c->dlam || !c->d_status || !c->d_occ || !c->d_bar) throw std::bad_alloc();
    if (cudaMemcpy(c->dB, c->B.data(), L * sizeof(double2*), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->dlam, c->lam.data(), (L + 1) * sizeof(double*), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(c->d_status, 0, sizeof(int)) != cudaSuccess ||
        cudaMemset(c->d_bar, 0, 4 * sizeof(unsigned int)) != cudaSuccess) {
      cudaGetLastError();
      tebd_destroy(c);
      return TEBD_ERR_CUDA;
    }
  } catch (...) {
    tebd_destroy(c);
    return TEBD_ERR_OOM;
  }
  *out = c;
  return TEBD_OK;
}

}  // namespace

extern "C" {

int tebd_create(int L, int n_max, int chi_max, double U, double J, double J_NNN, double K, double j_c, double dt,
                tebd_handle* out) {
  if (out) *out = nullptr;
  if (L < 3 || n_max < 1 || n_max > 7 || chi_max < 1) return TEBD_ERR_ARG;
  return create_impl(L, L, false, n_max, chi_max, U, J, J_NNN, K, j_c, dt, out);
}

int tebd_create_supersite(int L, int n_max, int chi_max, double U, double J, double J_NNN, double K, double j_c,
                          double dt, tebd_handle* out) {
  if (out) *out = nullptr;
  if (L < 3 || n_max < 1 || n_max > 4 || chi_max < 1) return TEBD_ERR_ARG;
  return create_impl((L + L % 2) / 2, L, true, n_max, chi_max, U, J, J_NNN, K, j_c, dt, out);
}

int tebd_set_option(tebd_handle h, const char* key, double value) {
  CHECK_HANDLE(h);
  if (key && std::string(key) == "graph_test_fallback") {  // diagnostic; keeps the cached graph
    if (value < 0 || value > 1000 || value != std::floor(value)) return TEBD_ERR_ARG;
    h->graph_test_fallback = (int)value;
    return TEBD_OK;
  }
  ++h->generation;  // a captured step holds the options it was captured with
  if (!key || !is_fin(value)) return TEBD_ERR_ARG;
  const std::string k(key);
  if (k == "w_cut") {
    if (value < 0 || value >= 1) return TEBD_ERR_ARG;
    h->w_cut = value;
  } else if (k == "eps_rel") {
    if (value < 0 || value >= 1) return TEBD_ERR_ARG;
    h->eps_rel = value;
  } else if (k == "precision") {
    if (value != 0.0 && value != 1.0 && value != 2.0) return TEBD_ERR_ARG;
    h->precision = (int)value;
  } else if (k == "trotter_order") {
    if (value != 2.0 && value != 4.0) return TEBD_ERR_ARG;
    if (h->ss && value != 2.0) return TEBD_ERR_ARG;  // the super-site split is second order
    if ((int)value != h->order) {
      if (h->stream && cudaStreamSynchronize(h->stream) != cudaSuccess) return fail_cuda(h);
      h->order = (int)value;
      if (int r = build_gates(h)) {
        h->sticky = r;
        return r;
      }
    }
  } else if (k == "profile") {
    if (value != 0.0 && value != 1.0) return TEBD_ERR_ARG;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail_cuda(h);
    prof_collect(h);
    h->prof = (value == 1.0);
    for (int q = 0; q < TEBD_PROF_NCLASS; ++q) {
      h->prof_ms[q] = 0.0;
      h->prof_launches[q] = 0;
      h->prof_work[q] = 0.0;
    }
  } else if (k == "randomized") {
    if (value != 0.0 && value != 1.0) return TEBD_ERR_ARG;
    if (value == 1.0 && (h->u1 || h->ss)) return TEBD_ERR_ARG;
    h->randomized = (value == 1.0);
  } else if (k == "oversample") {
    if (value < 0 || value > 4096 || value != std::floor(value)) return TEBD_ERR_ARG;
    h->oversample = (int)value;
  } else if (k == "power_iters") {
    if (value < 0 || value > 16 || value != std::floor(value)) return TEBD_ERR_ARG;
    h->power_iters = (int)value;
  } else if (k == "u1") {
    if (value != 0.0 && value != 1.0) return TEBD_ERR_ARG;
    if (value == 1.0 && (h->randomized || h->ss)) return TEBD_ERR_ARG;
    if ((value == 1.0) != h->u1) {
      if (!h->slots.empty()) return TEBD_ERR_STATE;  // the workspace is laid out for one form
      h->u1 = (value == 1.0);
    }
  } else if (k == "jacobi_max_sweeps") {
    if (value < 1 || value > 1000 || value != std::floor(value)) return TEBD_ERR_ARG;
    if ((int)value != h->jacobi_sweeps) {
      if (h->stream && cudaStreamSynchronize(h->stream) != cudaSuccess) return fail_cuda(h);
      h->jacobi_sweeps = (int)value;
      if (int r = build_gates(h)) {
        h->sticky = r;
        return r;
      }
    }
  } else if (k == "graph") {
    if (value != 0.0 && value != 1.0) return TEBD_ERR_ARG;
    if (value == 1.0 && (h->u1 || h->ss || h->randomized)) return TEBD_ERR_ARG;
    if (value == 1.0 && h->stream == nullptr) {
      // stream capture needs a stream other than the legacy one; a blocking stream stays
      // ordered with the legacy stream's other work
      if (!h->own_stream && cudaStreamCreate(&h->own_stream) != cudaSuccess) return fail_cuda(h);
      h->stream = h->own_stream;
    }
    h->graph = (value == 1.0);
    h->graph_broken = false;
  } else if (k == "panel_blocks") {
    if (value < 0 || value > 3 || value != std::floor(value)) return TEBD_ERR_ARG;
    h->panel_blocks = (int)value;
  } else if (k == "wait_limit_clocks") {
    if (value < 0 || value > 1e12 || value != std::floor(value)) return TEBD_ERR_ARG;
    h->wait_clocks = (long long)value;
  } else if (k == "max_slots") {
    if (value < 0 || value > MAX_SLOTS || value != std::floor(value)) return TEBD_ERR_ARG;
    if (!h->slots.empty()) return TEBD_ERR_STATE;
    h->max_slots = (int)value;
  } else {
    return TEBD_ERR_ARG;
  }
  return TEBD_OK;
}

int tebd_set_stream(tebd_handle h, void* cuda_stream) {
  CHECK_HANDLE(h);
  ++h->generation;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  return TEBD_OK;
}

int tebd_init_product(tebd_handle h, const int* occ) {
  CHECK_HANDLE(h);
  ++h->generation;
  if (!occ) return TEBD_ERR_ARG;
  const int n_occ = h->ss ? h->L_phys : h->L;
  for (int k = 0; k < n_occ; ++k)
    if (occ[k] < 0 || occ[k] > h->n_max) return TEBD_ERR_ARG;
  std::vector<int> sig(occ, occ + h->L);
  if (h->ss) {  // super site k holds physical sites (2k, 2k+1), sigma = s_a (n_max + 1) + s_b; a padded site is empty
    const int dp = h->n_max + 1;
    for (int k = 0; k < h->L; ++k)
      sig[k] = occ[2 * k] * dp + (2 * k + 1 < h->L_phys ? occ[2 * k + 1] : 0);
  }
  if (cudaMemcpyAsync(h->d_occ, sig.data(), h->L * sizeof(int), cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
    return fail_cuda(h);
  h->launches += launch_init_product(h->dB, h->dlam, h->d_occ, h->L, h->d, h->stream);
  if (int r = check_launch(h)) return r;
  if (int r = sync(h)) return r;  // occ is pageable caller memory
  std::fill(h->chi.begin(), h->chi.end(), 1);
  // bond charges of a product state: the boson count left of each bond
  h->q.assign(h->L + 1, std::vector<int>(1, 0));
  if (!h->ss)
    for (int k = 1; k <= h->L; ++k) h->q[k][0] = h->q[k - 1][0] + occ[k - 1];
  h->have_charges = !h->ss;
  h->steps = 0;
  h->w_total = 0.0;
  h->gate_updates = 0;
  h->have_state = true;
  return TEBD_OK;
}

int tebd_set_charges(tebd_handle h, const int* const* q_ptrs) {
  CHECK_HANDLE(h);
  if (!q_ptrs) return TEBD_ERR_ARG;
  if (!h->have_state) return TEBD_ERR_STATE;
  std::vector<std::vector<int>> q(h->L + 1);
  for (int k = 0; k <= h->L; ++k) {
    if (!q_ptrs[k]) return TEBD_ERR_ARG;
    q[k].assign(q_ptrs[k], q_ptrs[k] + h->chi[k]);
    for (int a = 0; a < h->chi[k]; ++a) {
      if (q[k][a] < 0 || q[k][a] > h->n_max * k) return TEBD_ERR_ARG;
      if (a > 0 && q[k][a] < q[k][a - 1]) return TEBD_ERR_ARG;  // each charge one contiguous run
    }
  }
  if (q[0][0] != 0) return TEBD_ERR_ARG;
  h->q.swap(q);
  h->have_charges = true;
  return TEBD_OK;
}

int tebd_set_test_matrices(tebd_handle h, tebd_test_matrix_fn fn, void* ctx) {
  CHECK_HANDLE(h);
  h->omega_fn = fn;
  h->omega_ctx = ctx;
  h->rcall = 0;
  return TEBD_OK;
}

int tebd_get_charges(tebd_handle h, int k, int* q) {
  CHECK_HANDLE(h);
  if (!q || k < 0 || k > h->L) return TEBD_ERR_ARG;
  if (!h->have_charges) return TEBD_ERR_STATE;
  std::copy(h->q[k].begin(), h->q[k].end(), q);
  return TEBD_OK;
}

int tebd_set_state(tebd_handle h, const int* chi, const double* const* B_ptrs, const double* const* lam_ptrs) {
  if (h) ++h->generation;
  CHECK_HANDLE(h);
  if (!chi || !B_ptrs || !lam_ptrs) return TEBD_ERR_ARG;
  if (chi[0] != 1 || chi[h->L] != 1) return TEBD_ERR_ARG;
  for (int k = 0; k <= h->L; ++k)
    if (chi[k] < 1 || chi[k] > h->cap[k]) return TEBD_ERR_ARG;
  for (int k = 0; k < h->L; ++k) {
    if (!B_ptrs[k]) return TEBD_ERR_ARG;
    const size_t n = (size_t)chi[k] * h->d * chi[k + 1];
    if (cudaMemcpy(h->B[k], B_ptrs[k], n * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess) return fail_cuda(h);
  }
  for (int k = 0; k <= h->L; ++k) {
    if (!lam_ptrs[k]) return TEBD_ERR_ARG;
    if (cudaMemcpy(h->lam[k], lam_ptrs[k], chi[k] * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail_cuda(h);
  }
  h->chi.assign(chi, chi + h->L + 1);
  h->have_charges = false;  // tebd_set_charges supplies them for the blocked form
  h->steps = 0;
  h->w_total = 0.0;
  h->gate_updates = 0;
  h->have_state = true;
  return TEBD_OK;
}

int tebd_step(tebd_handle h, int n_steps) {
  CHECK_HANDLE(h);
  if (n_steps < 0) return TEBD_ERR_ARG;
  if (!h->have_state || (h->u1 && !h->have_charges)) return TEBD_ERR_STATE;
  if (n_steps == 0) return TEBD_OK;
  try {
    if (int r = alloc_workspace(h)) return r;
    // the layers of one step (residue r <-> triples j = r+1 mod 3, gate-table index)
    const std::vector<std::pair<int, int>> layers = step_layers(h);
    const std::vector<tebd_ctx*> one{h};
    for (int n = 0; n < n_steps; ++n) {
      const int g = graph_step(h, one, layers);
      if (g < 0) return g;
      if (g == 1)
        for (const auto& l : layers)
          if (int r = run_layer(h, l.first, l.second)) return r;
      h->steps += 1;
    }
  } catch (...) {
    return TEBD_ERR_OOM;
  }
  return TEBD_OK;
}

int tebd_estimate_bytes(int L, int n_max, int chi_max, int max_slots, int precision, double* bytes) {
  if (!bytes || L < 3 || n_max < 1 || n_max > 7 || chi_max < 1 || max_slots < 0) return TEBD_ERR_ARG;
  if (precision < 0 || precision > 2) return TEBD_ERR_ARG;
  const int d = n_max + 1, D = d * d * d;
  const std::vector<int> cap = bond_caps(L, d, chi_max);
  double b = 0.0;
  long long capmax = 1;
  for (int k = 0; k < L; ++k) b += 16.0 * cap[k] * d * cap[k + 1];
  for (int k = 0; k <= L; ++k) {
    b += 8.0 * cap[k];
    capmax = std::max<long long>(capmax, cap[k]);
  }
  b += 16.0 * 2.0 * (L - 2) * (double)D * D;  // gates
  int slots = std::min(max_triples_per_layer(L), MAX_SLOTS);
  if (max_slots > 0) slots = std::min(slots, max_slots);
  b += slots * slot_bytes_for(capmax, d, chi_max, precision);
  b += 16.0 * MEAS_CHUNK * (2.0 * capmax * d * capmax + 2.0 * capmax * capmax) + 24.0 * L;  // measurement
  *bytes = b;
  return TEBD_OK;
}

int tebd_estimate_bytes_u1(int L, int n_max, int chi_max, int max_slots, int precision, double* bytes) {
  if (!bytes || L < 3 || n_max < 1 || n_max > 7 || chi_max < 1 || max_slots < 0) return TEBD_ERR_ARG;
  if (precision < 0 || precision > 2) return TEBD_ERR_ARG;
  const int d = n_max + 1, D = d * d * d;
  const std::vector<int> cap = bond_caps(L, d, chi_max);
  double b = 0.0;
  long long capmax = 1;
  for (int k = 0; k < L; ++k) b += 16.0 * cap[k] * d * cap[k + 1];  // dense site tensors
  for (int k = 0; k <= L; ++k) {
    b += 8.0 * cap[k];
    capmax = std::max<long long>(capmax, cap[k]);
  }
  b += 16.0 * 2.0 * (L - 2) * (double)D * D * 2.0;  // gate table and its occupation blocks (bounded by the table)
  int slots = std::min(max_triples_per_layer(L), MAX_SLOTS);
  if (max_slots > 0) slots = std::min(slots, max_slots);
  b += slots * U1_ARENA_FRACTION * 16.0 * (double)capmax * capmax * D;
  b += U1_RING_FRACTION * 16.0 * (double)capmax * capmax * D;  // exact-digit workspace rings
  b += 40.0 * L + 64.0e6;  // measurement buffers, staging
  *bytes = b;
  return TEBD_OK;
}

int tebd_batch_step(tebd_handle* hs, int n, int n_steps) {
  if (!hs || n < 1 || n_steps < 0) return TEBD_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    if (!hs[i]) return TEBD_ERR_ARG;
    if (hs[i]->sticky != TEBD_OK) return hs[i]->sticky;
    if (!hs[i]->have_state) return TEBD_ERR_STATE;
    if (hs[i]->device != hs[0]->device || hs[i]->precision != hs[0]->precision || hs[i]->order != hs[0]->order ||
        hs[i]->u1 != hs[0]->u1 || hs[i]->ss != hs[0]->ss || hs[i]->randomized != hs[0]->randomized)
      return TEBD_ERR_ARG;
    if (hs[i]->u1 && !hs[i]->have_charges) return TEBD_ERR_STATE;
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return TEBD_ERR_ARG;
  }
  if (n_steps == 0) return TEBD_OK;
  tebd_ctx* c = hs[0];
  std::vector<tebd_ctx*> v(hs, hs + n);
  int r = TEBD_OK;
  try {
    for (tebd_ctx* h : v)
      if ((r = alloc_workspace(h)) != TEBD_OK) return r;
    const std::vector<std::pair<int, int>> layers = step_layers(c);
    for (int step = 0; step < n_steps && r == TEBD_OK; ++step) {
      const int g = graph_step(c, v, layers);
      if (g < 0) r = g;
      for (size_t l = 0; g == 1 && l < layers.size() && r == TEBD_OK; ++l)
        r = run_layer_multi(c, v, layers[l].first, layers[l].second);
      if (r == TEBD_OK)
        for (tebd_ctx* h : v) h->steps += 1;
    }
  } catch (...) {
    r = TEBD_ERR_OOM;
  }
  if (r != TEBD_OK && c->sticky != TEBD_OK)  // a device error on the shared stream affects every member
    for (tebd_ctx* h : v) h->sticky = c->sticky;
  return r;
}

int tebd_layer(tebd_handle h, int residue, int full) {
  CHECK_HANDLE(h);
  if (residue < 0 || residue > (h->ss ? 1 : 2) || (full != 0 && full != 1)) return TEBD_ERR_ARG;
  if (h->order != 2) return TEBD_ERR_ARG;  // the gate table holds dt/2 and dt only at order 2
  if (!h->have_state || (h->u1 && !h->have_charges)) return TEBD_ERR_STATE;
  try {
    if (int r = alloc_workspace(h)) return r;
    return run_layer(h, residue, full);
  } catch (...) {
    return TEBD_ERR_OOM;
  }
}

}  // extern "C"

namespace {

// Observables of the super-site chain on its 2L physical sites: n of positions a and b of
// every super site; <b+ b> inside a super site (one-site term) and across a super bond
// (b+ on position b of k, b on position a of k + 1), the latter as the transfer
// products of the plain chain with the shifts of one position of the pair.
int measure_supersite(tebd_ctx* h, double* n_out, double* cur_out) {
  const int L = h->L, d = h->d, dp = h->n_max + 1, Lp = 2 * L;
  double mbytes = 0.0;
  for (int k = 0; k < L; ++k) mbytes += 16.0 * h->chi[k] * d * h->chi[k + 1];
  ProfScope ps(h, TEBD_PROF_MEASURE, 3.0 * mbytes);
  std::vector<DensityArgs> da(Lp);
  for (int k = 0; k < L; ++k)
    for (int pos = 0; pos < 2; ++pos)
      da[2 * k + pos] = DensityArgs{h->B[k], h->lam[k], h->mN + 2 * k + pos, h->chi[k], d, h->chi[k + 1], 1 + pos, dp};
  h->launches += launch_densities(da.data(), Lp, h->stream);
  for (int k = 0; k < L; ++k)
    h->launches += launch_pair_hop(h->B[k], h->lam[k], h->chi[k], d, h->chi[k + 1], dp, h->mC + 2 * k, h->stream);
  const long long capmax = std::max<long long>(1, *std::max_element(h->cap.begin(), h->cap.end()));
  const long long big = capmax * d * capmax;
  for (int k0 = 0; k0 < L - 1; k0 += MEAS_CHUNK) {
    const int k1 = std::min(L - 1, k0 + MEAS_CHUNK);
    Gemm gx(true, OP_C, OP_N), gy(true, OP_N, OP_C);
    for (int k = k0; k < k1; ++k) {
      const int q = k - k0;
      const int cl = h->chi[k], cm = h->chi[k + 1], cr = h->chi[k + 2];
      double2* P = h->mP + q * big;
      double2* Q = h->mQ + q * big;
      // b+ on position b of super site k (sigma -> sigma + 1), b on position a of k + 1 (sigma -> sigma - dp)
      h->launches += launch_shift_pair(h->B[k], h->lam[k], P, cl, d, cm, 1, 1, dp, h->stream);
      h->launches += launch_shift_pair(h->B[k + 1], nullptr, Q, cm, d, cr, dp, 2, dp, h->stream);
      gx.add(cm, cm, cl * d, P, cm, h->B[k], cm, h->mX + q * capmax * capmax, cm);
      gy.add(cm, cm, d * cr, Q, (long long)d * cr, h->B[k + 1], (long long)d * cr, h->mY + q * capmax * capmax, cm);
    }
    h->launches += gx.launch(h->stream);
    h->launches += gy.launch(h->stream);
    for (int k = k0; k < k1; ++k) {
      const int q = k - k0;
      h->launches += launch_trace_product(h->mX + q * capmax * capmax, h->mY + q * capmax * capmax, h->chi[k + 1],
                                          h->mC + 2 * k + 1, h->stream);
    }
  }
  if (int r = check_launch(h)) return r;
  if (int r = ensure_pinned(h, 3 * (size_t)Lp + 8)) return r;
  cudaMemcpyAsync(h->h_pinned, h->mN, Lp * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  cudaMemcpyAsync(h->h_pinned + Lp, h->mC, (Lp - 1) * sizeof(double2), cudaMemcpyDeviceToHost, h->stream);
  if (int r = sync(h)) return r;
  if (n_out) std::memcpy(n_out, h->h_pinned, Lp * sizeof(double));
  if (cur_out)
    for (int j = 0; j < Lp - 1; ++j) cur_out[j] = 2.0 * h->J * h->h_pinned[Lp + 2 * j + 1];
  return TEBD_OK;
}

}  // namespace

extern "C" {

int tebd_measure(tebd_handle h, double* n_out, double* cur_out) {
  CHECK_HANDLE(h);
  if (!h->have_state) return TEBD_ERR_STATE;
  try {
    if (int r = ensure_measure_ws(h)) return r;
    if (h->ss) return measure_supersite(h, n_out, cur_out);
    const int L = h->L, d = h->d;
    double mbytes = 0.0;
    for (int k = 0; k < L; ++k) mbytes += 16.0 * h->chi[k] * d * h->chi[k + 1];
    ProfScope ps(h, TEBD_PROF_MEASURE, mbytes);
    std::vector<DensityArgs> da(L);
    for (int k = 0; k < L; ++k) da[k] = DensityArgs{h->B[k], h->lam[k], h->mN + k, h->chi[k], d, h->chi[k + 1]};
    h->launches += launch_densities(da.data(), L, h->stream);
    const long long capmax = std::max<long long>(1, *std::max_element(h->cap.begin(), h->cap.end()));
    const long long big = capmax * d * capmax;
    if (h->u1 && h->have_charges) {  // the correlators from the charge blocks
      if (!h->u1w)
        if (int r = u1_alloc_slots(h, 0)) return r;
      if (int r = u1_correlators(h, h->mC)) return r;
    }
    for (int k0 = 0; k0 < (h->u1 && h->have_charges ? 0 : L - 1); k0 += MEAS_CHUNK) {
      const int k1 = std::min(L - 1, k0 + MEAS_CHUNK);
      Gemm gx(true, OP_C, OP_N), gy(true, OP_N, OP_C);
      for (int k = k0; k < k1; ++k) {
        const int q = k - k0;
        const int cl = h->chi[k], cm = h->chi[k + 1], cr = h->chi[k + 2];
        double2* P = h->mP + q * big;
        double2* Q = h->mQ + q * big;
        h->launches += launch_shift_left(h->B[k], h->lam[k], P, cl, d, cm, h->stream);
        h->launches += launch_shift_right(h->B[k + 1], Q, cm, d, cr, h->stream);
        gx.add(cm, cm, cl * d, P, cm, h->B[k], cm, h->mX + q * capmax * capmax, cm);
        gy.add(cm, cm, d * cr, Q, (long long)d * cr, h->B[k + 1], (long long)d * cr, h->mY + q * capmax * capmax, cm);
      }
      h->launches += gx.launch(h->stream);
      h->launches += gy.launch(h->stream);
      for (int k = k0; k < k1; ++k) {
        const int q = k - k0;
        h->launches += launch_trace_product(h->mX + q * capmax * capmax, h->mY + q * capmax * capmax, h->chi[k + 1],
                                            h->mC + k, h->stream);
      }
    }
    if (int r = check_launch(h)) return r;
    if (int r = ensure_pinned(h, 3 * (size_t)L + 8)) return r;
    cudaMemcpyAsync(h->h_pinned, h->mN, L * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    cudaMemcpyAsync(h->h_pinned + L, h->mC, (L - 1) * sizeof(double2), cudaMemcpyDeviceToHost, h->stream);
    int* h_status = reinterpret_cast<int*>(h->h_pinned + 3 * (size_t)L);  // the tensor-core waits' status
    cudaMemcpyAsync(h_status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (int r = sync(h)) return r;
    if (*h_status != 0) {
      h->sticky = *h_status;
      return *h_status;
    }
    if (n_out) std::memcpy(n_out, h->h_pinned, L * sizeof(double));
    if (cur_out)
      for (int k = 0; k < L - 1; ++k) cur_out[k] = 2.0 * h->J * h->h_pinned[L + 2 * k + 1];
  } catch (...) {
    return TEBD_ERR_OOM;
  }
  return TEBD_OK;
}

int tebd_device_bytes(tebd_handle h, double* bytes) {
  CHECK_HANDLE(h);
  if (!bytes) return TEBD_ERR_ARG;
  *bytes = (double)(h->alloc_bytes + h->Gblk_n * sizeof(double2) + u1_workspace_bytes(h));
  return TEBD_OK;
}

int tebd_stats(tebd_handle h, double* t, double* w_total, int* max_chi) {
  CHECK_HANDLE(h);
  if (t) *t = (double)h->steps * h->dt;
  if (w_total) *w_total = h->w_total;
  if (max_chi) *max_chi = *std::max_element(h->chi.begin(), h->chi.end());
  return TEBD_OK;
}

int tebd_bond_dims(tebd_handle h, int* chi) {
  CHECK_HANDLE(h);
  if (!chi) return TEBD_ERR_ARG;
  std::copy(h->chi.begin(), h->chi.end(), chi);
  return TEBD_OK;
}

int tebd_get_site(tebd_handle h, int k, double* B, double* lam) {
  CHECK_HANDLE(h);
  if (k < 0 || k > h->L) return TEBD_ERR_ARG;
  if (B && k == h->L) return TEBD_ERR_ARG;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail_cuda(h);
  if (B) {
    const size_t n = (size_t)h->chi[k] * h->d * h->chi[k + 1];
    if (cudaMemcpy(B, h->B[k], n * sizeof(double2), cudaMemcpyDeviceToHost) != cudaSuccess) return fail_cuda(h);
  }
  if (lam && cudaMemcpy(lam, h->lam[k], h->chi[k] * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail_cuda(h);
  return TEBD_OK;
}

int tebd_profile(tebd_handle h, int cls, double* ms, long long* launches, double* work) {
  CHECK_HANDLE(h);
  if (cls < 0 || cls >= TEBD_PROF_NCLASS) return TEBD_ERR_ARG;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail_cuda(h);
  prof_collect(h);
  if (ms) *ms = h->prof_ms[cls];
  if (launches) *launches = h->prof_launches[cls];
  if (work) *work = h->prof_work[cls];
  return TEBD_OK;
}

int tebd_counters(tebd_handle h, long long* gate_updates, long long* kernel_launches) {
  CHECK_HANDLE(h);
  if (gate_updates) *gate_updates = h->gate_updates;
  if (kernel_launches) *kernel_launches = h->launches;
  return TEBD_OK;
}

void tebd_destroy(tebd_handle h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  prof_collect(h);
  for (cudaEvent_t e : h->event_pool) cudaEventDestroy(e);
  u1_release(h);
  if (h->Gblk) cudaFree(h->Gblk);
  for (void* p : h->allocs) cudaFree(p);
  if (h->h_pinned) cudaFreeHost(h->h_pinned);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->h_gw) cudaFreeHost(h->h_gw);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  cudaGetLastError();
  delete h;
}

int tebd_graph_stats(tebd_handle h, long long* replays, long long* fallbacks, long long* launches_per_replay) {
  CHECK_HANDLE(h);
  if (replays) *replays = h->graph_replays;
  if (fallbacks) *fallbacks = h->graph_fallbacks;
  if (launches_per_replay) *launches_per_replay = h->gexec ? h->glaunches : 0;
  return TEBD_OK;
}

}  // extern "C"
