// Daubechies orthonormal low-pass filters DbK (K vanishing moments, 2K taps),
// built at load time in long double from the spectral factorisation:
//   |m0(w)|^2 = cos^{2K}(w/2) P(sin^2(w/2)),  P(y) = sum_{k<K} C(K-1+k, k) y^k.
// Each root y of P gives a pair of zeros z, 1/z of z^2 - (2 - 4y) z + 1; the
// extremal-phase filter keeps the zero outside the unit circle of
// H(z) = sum_n h_n z^n (Daubechies 1988; the wavelet dictionary of the
// paper's Section 4 is Db1..Db8 and Haar).  The roots of P are found with the
// Durand-Kerner (Weierstrass) simultaneous iteration.
#include <cmath>
#include <complex>

#include "mf_internal.cuh"

namespace mf {

typedef long double ld;
typedef std::complex<ld> cld;

static ld binom(int n, int k) {
  ld r = 1;
  for (int i = 1; i <= k; i++) r = r * (ld)(n - k + i) / (ld)i;
  return r;
}

static cld poly_eval(const ld* c, int deg, cld z) {  // c: increasing powers
  cld acc = c[deg];
  for (int i = deg - 1; i >= 0; i--) acc = acc * z + c[i];
  return acc;
}

static void daubechies(int K, double* h) {
  if (K == 1) {
    h[0] = h[1] = (double)std::sqrt((ld)0.5);
    return;
  }
  const int deg = K - 1;
  ld c[MF_MAX_K];
  for (int k = 0; k <= deg; k++) c[k] = binom(K - 1 + k, k);
  // monic copy for the iteration
  ld m[MF_MAX_K];
  for (int k = 0; k <= deg; k++) m[k] = c[k] / c[deg];
  cld r[MF_MAX_K];
  const cld seed((ld)0.4, (ld)0.9);
  cld p = 1;
  for (int i = 0; i < deg; i++) { r[i] = p; p *= seed; }
  for (int it = 0; it < 2000; it++) {
    ld change = 0;
    for (int i = 0; i < deg; i++) {
      cld den = 1;
      for (int j = 0; j < deg; j++)
        if (j != i) den *= (r[i] - r[j]);
      cld d = poly_eval(m, deg, r[i]) / den;
      r[i] -= d;
      change = std::fmax(change, std::abs(d));
    }
    if (change < 1e-30L) break;
  }
  // zeros in z outside the unit circle
  cld q[2 * MF_MAX_K];
  int qd = 0;
  q[0] = 1;
  for (int i = 0; i < deg; i++) {
    cld b = (ld)1 - (ld)2 * r[i];
    cld disc = std::sqrt(b * b - (ld)1);
    cld z1 = b + disc, z2 = b - disc;
    cld z = std::abs(z1) > 1 ? z1 : z2;
    // q <- q * (x - z)
    q[qd + 1] = 0;
    for (int k = qd + 1; k >= 1; k--) q[k] = q[k - 1] - z * q[k];
    q[0] = -z * q[0];
    qd++;
  }
  // multiply by (1 + z)^K
  ld hp[2 * MF_MAX_K] = {0};
  for (int a = 0; a <= qd; a++)
    for (int n = 0; n <= K; n++) hp[a + n] += q[a].real() * binom(K, n);
  ld s = 0;
  for (int n = 0; n < 2 * K; n++) s += hp[n];
  for (int n = 0; n < 2 * K; n++) h[n] = (double)(hp[n] * std::sqrt((ld)2) / s);
}

namespace {
struct TapTable {
  double taps[MF_MAX_K + 1][2 * MF_MAX_K];
  TapTable() {
    for (int k = 1; k <= MF_MAX_K; k++) daubechies(k, taps[k]);
  }
};
}  // namespace

const double* filter_taps(int K) {
  static const TapTable table;  // initialised once, thread-safe
  return table.taps[K];
}

}  // namespace mf
