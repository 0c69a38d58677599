// Host-side FP64 gate construction: G_j(tau) = exp(-i h_j tau).
//
// h_j is the three-site share of the Hamiltonian of eq. (1) (Sec. I A) on the
// triple (j, j+1, j+2): the NNN hop of the triple, each NN hop inside it
// divided by the number of triples containing that bond, and each on-site
// term divided by the number of triples containing that site, so that
// sum_j h_j reproduces eq. (1) exactly.  The second-order Trotter gates of
// Sec. II B are exact exponentials of these local terms; the exponential is
// taken through a cyclic complex Jacobi eigen-decomposition h = V E V^+.
#include "ptebd_internal.h"

#include <cmath>
#include <algorithm>
#include <complex>
#include <vector>

namespace ptebd {

using cd = std::complex<double>;

namespace {

int triples_with_bond(int k, int L) {  // bond (k, k+1), 1-based
  int c = 0;
  for (int j = k - 1; j <= k; ++j) c += (j >= 1 && j <= L - 2);
  return c;
}

int triples_with_site(int k, int L) {  // site k, 1-based
  int c = 0;
  for (int j = k - 2; j <= k; ++j) c += (j >= 1 && j <= L - 2);
  return c;
}

// Cyclic Jacobi for a Hermitian n x n matrix A (row-major, overwritten).
// On return E holds the eigenvalues and V (row-major) the eigenvectors as
// columns.  Each rotation first removes the phase of a_pq, then applies the
// real rotation that zeroes it.
bool hermitian_jacobi(int n, std::vector<cd>& A, std::vector<double>& E, std::vector<cd>& V, int max_sweeps) {
  V.assign((size_t)n * n, cd(0, 0));
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  double fro = 0;
  for (auto& x : A) fro += std::norm(x);
  bool converged = false;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    double off = 0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += std::norm(A[(size_t)p * n + q]);
    if (off <= 1e-32 * fro || off == 0.0) { converged = true; break; }
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        cd apq = A[(size_t)p * n + q];
        double g = std::abs(apq);
        if (g == 0.0) continue;
        double app = A[(size_t)p * n + p].real(), aqq = A[(size_t)q * n + q].real();
        cd ph = apq / g;  // e^{i phi}
        double theta = (aqq - app) / (2.0 * g);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        cd phc = std::conj(ph);
        // columns: A <- A J, J = [[c, s], [-s e^{-i phi}, c e^{-i phi}]] on (p, q)
        for (int r = 0; r < n; ++r) {
          cd xp = A[(size_t)r * n + p], xq = A[(size_t)r * n + q];
          A[(size_t)r * n + p] = c * xp - s * phc * xq;
          A[(size_t)r * n + q] = s * xp + c * phc * xq;
          cd vp = V[(size_t)r * n + p], vq = V[(size_t)r * n + q];
          V[(size_t)r * n + p] = c * vp - s * phc * vq;
          V[(size_t)r * n + q] = s * vp + c * phc * vq;
        }
        // rows: A <- J^+ A
        for (int cix = 0; cix < n; ++cix) {
          cd xp = A[(size_t)p * n + cix], xq = A[(size_t)q * n + cix];
          A[(size_t)p * n + cix] = c * xp - s * ph * xq;
          A[(size_t)q * n + cix] = s * xp + c * ph * xq;
        }
        A[(size_t)p * n + q] = 0.0;
        A[(size_t)q * n + p] = 0.0;
      }
    }
  }
  E.resize(n);
  for (int i = 0; i < n; ++i) E[i] = A[(size_t)i * n + i].real();
  return converged;
}

}  // namespace

// Three-site term h_j (1-based j) as a D x D row-major complex matrix, D = d^3.
std::vector<cd> three_site_term(int L, int n_max, double U, double J, double Jnnn, double K,
                                double jc, int j) {
  const int d = n_max + 1, D = d * d * d;
  std::vector<cd> h((size_t)D * D, cd(0, 0));
  for (int a = 0; a < D; ++a) {
    int n[3] = {a / (d * d), (a / d) % d, a % d};
    double diag = 0;
    for (int p = 0; p < 3; ++p) {
      int k = j + p;
      double x = k - jc;
      diag += (0.5 * U * n[p] * (n[p] - 1) + 0.5 * K * x * x * n[p]) / triples_with_site(k, L);
    }
    h[(size_t)a * D + a] += diag;
    // hops b+_p b_q on positions (p, q): NN pairs (0,1), (1,2) shared; NNN pair (0,2)
    const int pairs[3][2] = {{0, 1}, {1, 2}, {0, 2}};
    for (int e = 0; e < 3; ++e) {
      int p0 = pairs[e][0], q0 = pairs[e][1];
      double amp0 = (e < 2) ? -J / triples_with_bond(j + p0, L) : -Jnnn;
      for (int dir = 0; dir < 2; ++dir) {
        int p = dir ? q0 : p0, q = dir ? p0 : q0;  // b+_p b_q
        if (n[q] == 0 || n[p] == n_max) continue;
        int m[3] = {n[0], n[1], n[2]};
        double amp = std::sqrt((double)(m[p] + 1) * m[q]);
        m[p] += 1;
        m[q] -= 1;
        int b = (m[0] * d + m[1]) * d + m[2];
        h[(size_t)b * D + a] += amp0 * amp;
      }
    }
  }
  return h;
}

bool build_gate(int L, int n_max, double U, double J, double Jnnn, double K, double jc, int j,
                double tau, std::vector<cd>& G, int max_sweeps) {
  const int d = n_max + 1, D = d * d * d;
  std::vector<cd> h = three_site_term(L, n_max, U, J, Jnnn, K, jc, j);
  std::vector<double> E;
  std::vector<cd> V;
  bool ok = hermitian_jacobi(D, h, E, V, max_sweeps);
  G.assign((size_t)D * D, cd(0, 0));
  std::vector<cd> ph(D);
  for (int k = 0; k < D; ++k) ph[k] = std::exp(cd(0, -E[k] * tau));
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c) {
      cd acc(0, 0);
      for (int k = 0; k < D; ++k) acc += V[(size_t)r * D + k] * ph[k] * std::conj(V[(size_t)c * D + k]);
      G[(size_t)r * D + c] = acc;
    }
  return ok;
}

// ---- super sites (pairs of physical sites, the paper's scheme of Sec. II B) ----------------
// Super site k (1-based) holds physical sites 2k-1 and 2k of the chain padded to even
// length L' = L + (L mod 2); its basis index is sigma = s_a d + s_b.  The term of super
// bond (k, k+1) acts on physical sites 2k-1 .. 2k+2 (positions 0..3, position 3 fastest):
// the couplings between the two super sites (NN hop of positions 1, 2; NNN hops 0-2 and
// 1-3) in full, and the terms inside each super site (its NN hop and on-site terms)
// divided by the number of super bonds that contain it, so that the bond terms sum to
// eq. (1) on the padded chain.
std::vector<cd> supersite_bond_term(int L, int n_max, double U, double J, double Jnnn, double K, double jc, int k) {
  const int d = n_max + 1, D = d * d * d * d;
  const int Lp = L + (L % 2), Le = Lp / 2;
  std::vector<cd> h((size_t)D * D, cd(0, 0));
  auto mult = [&](int kk) { return (kk >= 2 ? 1 : 0) + (kk <= Le - 1 ? 1 : 0); };
  for (int a = 0; a < D; ++a) {
    int n[4] = {a / (d * d * d), (a / (d * d)) % d, (a / d) % d, a % d};
    double diag = 0;
    for (int pos = 0; pos < 4; ++pos) {
      const int kk = (pos < 2) ? k : k + 1;
      const int site = 2 * kk - 1 + (pos % 2);
      const double x = site - jc;
      diag += (0.5 * U * n[pos] * (n[pos] - 1) + 0.5 * K * x * x * n[pos]) / mult(kk);
    }
    h[(size_t)a * D + a] += diag;
    // hops b+_p b_q + h.c.: (position pair, amplitude)
    const int pairs[5][2] = {{1, 2}, {0, 2}, {1, 3}, {0, 1}, {2, 3}};
    const double amps[5] = {-J, -Jnnn, -Jnnn, -J / mult(k), -J / mult(k + 1)};
    for (int e = 0; e < 5; ++e) {
      for (int dir = 0; dir < 2; ++dir) {
        const int p = dir ? pairs[e][1] : pairs[e][0], q = dir ? pairs[e][0] : pairs[e][1];  // b+_p b_q
        if (n[q] == 0 || n[p] == n_max) continue;
        int m[4] = {n[0], n[1], n[2], n[3]};
        const double amp = std::sqrt((double)(m[p] + 1) * m[q]);
        m[p] += 1;
        m[q] -= 1;
        const int b = ((m[0] * d + m[1]) * d + m[2]) * d + m[3];
        h[(size_t)b * D + a] += amps[e] * amp;
      }
    }
  }
  return h;
}

// G = exp(-i h tau) for a Hermitian h that conserves the total occupation (occ[x] of basis
// state x): each occupation block diagonalised on its own by the cyclic Jacobi solver.
bool exp_by_occupation(const std::vector<cd>& h, const std::vector<int>& occ, double tau, std::vector<cd>& G,
                       int max_sweeps) {
  const int D = (int)occ.size();
  G.assign((size_t)D * D, cd(0, 0));
  const int nmax = *std::max_element(occ.begin(), occ.end());
  bool ok = true;
  for (int t = 0; t <= nmax; ++t) {
    std::vector<int> mem;
    for (int x = 0; x < D; ++x)
      if (occ[x] == t) mem.push_back(x);
    const int n = (int)mem.size();
    if (n == 0) continue;
    std::vector<cd> A((size_t)n * n), V;
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) A[(size_t)r * n + c] = h[(size_t)mem[r] * D + mem[c]];
    std::vector<double> E;
    ok = hermitian_jacobi(n, A, E, V, max_sweeps) && ok;
    std::vector<cd> ph(n);
    for (int q = 0; q < n; ++q) ph[q] = std::exp(cd(0, -E[q] * tau));
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) {
        cd acc(0, 0);
        for (int q = 0; q < n; ++q) acc += V[(size_t)r * n + q] * ph[q] * std::conj(V[(size_t)c * n + q]);
        G[(size_t)mem[r] * D + mem[c]] = acc;
      }
  }
  return ok;
}

bool build_gate_supersite(int L, int n_max, double U, double J, double Jnnn, double K, double jc, int k, double tau,
                          std::vector<cd>& G, int max_sweeps) {
  const int d = n_max + 1, D = d * d * d * d;
  std::vector<cd> h = supersite_bond_term(L, n_max, U, J, Jnnn, K, jc, k);
  std::vector<int> occ(D);
  for (int x = 0; x < D; ++x) occ[x] = x / (d * d * d) + (x / (d * d)) % d + (x / d) % d + x % d;
  return exp_by_occupation(h, occ, tau, G, max_sweeps);
}

}  // namespace ptebd
