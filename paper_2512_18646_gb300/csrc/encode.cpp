// encode.cpp - CKKS canonical-embedding encode / decode on the host.
//
// Slot j of a message corresponds to the root zeta^(5^j mod 2N), zeta =
// exp(i pi / N), j < M = N/2; a real message polynomial m has m(zeta^(5^j)) =
// scale * z_j (Cheon et al. 2017, the CKKS scheme of Sec. II-A).
//
// Route taken here: with w_k = m_k + i m_{k+M} (k < M), and zeta^(5^j M) = i,
//   m(zeta^(5^j)) = w(zeta^(5^j)) = sum_k (w_k zeta^k) omega^(t_j k),
// omega = zeta^4 = exp(2 pi i / M), t_j = (5^j mod 2N - 1) / 4. So decoding is
// a twist by zeta^k followed by an M-point DFT read at t_j, and encoding is the
// inverse: place z_j at t_j, inverse M-point DFT, untwist, split real and
// imaginary parts into m_k and m_{k+M}, round to nearest (ties away from zero).
#include <cmath>
#include <complex>
#include <vector>

#include "he_internal.h"

namespace he {

typedef std::complex<double> cd;

// In-place iterative radix-2 DFT of length M (a power of two) with the
// context's roots exp(2 pi i k / M); sign +1 or -1 selects the exponent sign.
static void dft(const Ctx& C, std::vector<cd>& a, int sign) {
  const size_t M = a.size();
  int bits = 0;
  while (((size_t)1 << bits) < M) bits++;
  for (size_t i = 1, j = 0; i < M; i++) {
    size_t bit = M >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  const double* R = C.fft_root.data();
  for (size_t len = 2; len <= M; len <<= 1) {
    const size_t step = M / len, half = len / 2;
    for (size_t i = 0; i < M; i += len) {
      for (size_t k = 0; k < half; k++) {
        const size_t r = k * step;
        const cd w(R[2 * r], sign * R[2 * r + 1]);
        const cd u = a[i + k], v = a[i + k + half] * w;
        a[i + k] = u + v;
        a[i + k + half] = u - v;
      }
    }
  }
}

void encode_real(const Ctx& C, const double* z, size_t nz, double scale, int64_t* m) {
  const size_t M = C.N / 2;
  if (nz > M) throw Error(1, "more values than slots");
  std::vector<cd> y(M, cd(0.0, 0.0));
  for (size_t j = 0; j < nz; j++) y[C.slot_index[j]] = cd(z[j], 0.0);
  dft(C, y, -1);
  const double inv_m = 1.0 / (double)M;
  for (size_t k = 0; k < M; k++) {
    const cd untwist(C.fft_twist[2 * k], -C.fft_twist[2 * k + 1]);
    const cd w = y[k] * untwist * inv_m;
    m[k] = std::llround(w.real() * scale);
    m[k + M] = std::llround(w.imag() * scale);
  }
}

void decode_real(const Ctx& C, const double* m, double scale, double* z) {
  const size_t M = C.N / 2;
  std::vector<cd> u(M);
  for (size_t k = 0; k < M; k++) u[k] = cd(m[k], m[k + M]) * cd(C.fft_twist[2 * k], C.fft_twist[2 * k + 1]);
  dft(C, u, +1);
  for (size_t j = 0; j < M; j++) z[j] = u[C.slot_index[j]].real() / scale;
}

}  // namespace he
