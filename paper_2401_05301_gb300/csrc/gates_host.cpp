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

}  // namespace ptebd
