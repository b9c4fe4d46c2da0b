// The Chebyshev polynomial basis that Section 4 suggests for the spectral
// dictionary W_nu, made orthonormal on the L equispaced bands: the discrete
// Chebyshev (Gram) polynomials p_n on x = 0..L-1, row n of the matrix, degree
// n, positive leading coefficient.
//
// They are computed as the eigenvectors of their difference equation, the
// Hahn equation with alpha = beta = 0 (N = L - 1):
//   n(n+1) p(x) = B(x) p(x+1) - (B(x) + D(x)) p(x) + D(x) p(x-1),
//   B(x) = (x+1)(x-N),  D(x) = x(x-N-1),
// whose matrix is symmetric tridiagonal (B(x) = D(x+1)) with the distinct
// eigenvalues n(n+1), n = 0..N: well separated (gaps >= 2), so the
// eigenvectors are well determined.  The three-term recurrence in n, by
// contrast, loses all accuracy for large n at L = 64.  The eigenproblem is
// solved by cyclic Jacobi rotations in long double; each eigenvector is
// normalised and signed so that p_n(N) > 0 (a polynomial with positive leading
// coefficient is positive beyond its largest zero, which lies inside (0, N)).
#include <algorithm>
#include <cmath>
#include <vector>

#include "mf_internal.cuh"

namespace mf {

void chebyshev_matrix(int L, double* out) {
  typedef long double ld;
  const int n = L;
  const ld N = (ld)(L - 1);
  std::vector<ld> A((size_t)n * n, 0.0L), V((size_t)n * n, 0.0L);
  for (int x = 0; x < n; x++) {
    const ld B = ((ld)x + 1.0L) * ((ld)x - N), D = (ld)x * ((ld)x - N - 1.0L);
    A[(size_t)x * n + x] = -(B + D);
    if (x + 1 < n) A[(size_t)x * n + x + 1] = A[(size_t)(x + 1) * n + x] = B;
    V[(size_t)x * n + x] = 1.0L;
  }
  for (int sweep = 0; sweep < 64; sweep++) {
    ld off = 0.0L, diag = 0.0L;
    for (int p = 0; p < n; p++)
      for (int q = 0; q < n; q++) (p == q ? diag : off) += A[(size_t)p * n + q] * A[(size_t)p * n + q];
    if (off <= 1e-36L * diag) break;
    for (int p = 0; p < n; p++)
      for (int q = p + 1; q < n; q++) {
        const ld apq = A[(size_t)p * n + q];
        if (apq == 0.0L) continue;
        const ld theta = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0L * apq);
        const ld t = (theta >= 0 ? 1.0L : -1.0L) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0L));
        const ld c = 1.0L / std::sqrt(t * t + 1.0L), s = t * c;
        for (int k = 0; k < n; k++) {  // columns p, q
          const ld akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - s * akq;
          A[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; k++) {  // rows p, q
          const ld apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - s * aqk;
          A[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; k++) {  // eigenvector columns
          const ld vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  // order by eigenvalue (degree), normalise, sign by the value at x = N
  std::vector<int> order(n);
  for (int i = 0; i < n; i++) order[i] = i;
  std::sort(order.begin(), order.end(),
            [&](int a, int b) { return A[(size_t)a * n + a] < A[(size_t)b * n + b]; });
  for (int deg = 0; deg < n; deg++) {
    const int j = order[deg];
    ld norm = 0.0L;
    for (int x = 0; x < n; x++) norm += V[(size_t)x * n + j] * V[(size_t)x * n + j];
    ld sc = 1.0L / std::sqrt(norm);
    if (V[(size_t)(n - 1) * n + j] < 0) sc = -sc;
    for (int x = 0; x < n; x++) out[(size_t)deg * n + x] = (double)(V[(size_t)x * n + j] * sc);
  }
}

}  // namespace mf
