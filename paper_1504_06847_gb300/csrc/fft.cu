// Step I of Algorithm 1 (Eqs. linsystemX, matQ, Qlsimp): per band
//   x_l = Q_l^-1 b_l,  Q_l = H_l^T H_l + rho I,
// solved in the Fourier domain as X = c + g F(b_rest) with
//   g = 1 / ((|h|^2 + rho) N^2),  c = conj(h) F(y) g
// (the paper's filter with frequency response (|h_l|^2 + rho)^-1, Section 3;
// the H^T y term of Eq. matB folded into c, the 1/N^2 of the inverse into both).
//
// Three shared-memory Stockham passes per iteration:
//   rows_fwd : real rows -> packed half spectrum (N/2 complex per row; the
//              real-valued Nyquist bin rides in the imaginary part of bin 0)
//   cols     : column FFT of a strip of packed columns, the divide, the
//              inverse column FFT, all in one CTA; column 0 carries the DC and
//              Nyquist columns as one complex column and is unpacked through
//              its Hermitian symmetry for the divide
//   rows_inv : packed half spectrum -> real rows
// Every FFT is a mixed-radix Stockham transform (one radix-2/4 pass, then
// radix-8 passes; Govindaraju et al., SC'08) with the butterflies' operands in
// registers and the exchange through one shared buffer.
#include <cuda_runtime.h>

#include "mf_internal.cuh"
#include "reduce.cuh"

namespace mf {

template <class R> __device__ __forceinline__ cx<R> mk(R x, R y) { cx<R> c; c.x = x; c.y = y; return c; }
template <class R> __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return mk<R>(a.x + b.x, a.y + b.y); }
template <class R> __device__ __forceinline__ cx<R> cadd(cx<R> a, cx<R> b) { return mk<R>(a.x + b.x, a.y + b.y); }
template <class R> __device__ __forceinline__ cx<R> csub(cx<R> a, cx<R> b) { return mk<R>(a.x - b.x, a.y - b.y); }
template <class R> __device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
  return mk<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <class R> __device__ __forceinline__ cx<R> cconj(cx<R> a) { return mk<R>(a.x, -a.y); }
template <class R> __device__ __forceinline__ cx<R> cscale(cx<R> a, R s) { return mk<R>(a.x * s, a.y * s); }

// ---------------------------------------------------------------------------
// Small forward DFTs in registers (kernel e^{-2 pi i / RAD}).
// ---------------------------------------------------------------------------
template <class R, int RAD> struct Dft;
template <class R> struct Dft<R, 2> {
  static __device__ __forceinline__ void run(cx<R>* v) {
    cx<R> a = v[0], b = v[1];
    v[0] = cadd<R>(a, b);
    v[1] = csub<R>(a, b);
  }
};
template <class R> struct Dft<R, 4> {
  static __device__ __forceinline__ void run(cx<R>* v) {
    cx<R> s02 = cadd<R>(v[0], v[2]), d02 = csub<R>(v[0], v[2]);
    cx<R> s13 = cadd<R>(v[1], v[3]), d13 = csub<R>(v[1], v[3]);
    v[0] = cadd<R>(s02, s13);
    v[2] = csub<R>(s02, s13);
    v[1] = mk<R>(d02.x + d13.y, d02.y - d13.x);  // d02 - i d13
    v[3] = mk<R>(d02.x - d13.y, d02.y + d13.x);  // d02 + i d13
  }
};
template <class R> struct Dft<R, 8> {
  static __device__ __forceinline__ void run(cx<R>* v) {
    const R s = (R)0.70710678118654752440084436210485;
    cx<R> b[4], c[4];
#pragma unroll
    for (int t = 0; t < 4; t++) {
      b[t] = cadd<R>(v[t], v[t + 4]);
      c[t] = csub<R>(v[t], v[t + 4]);
    }
    c[1] = mk<R>(s * (c[1].x + c[1].y), s * (c[1].y - c[1].x));   // * e^{-i pi/4}
    c[2] = mk<R>(c[2].y, -c[2].x);                                  // * -i
    c[3] = mk<R>(s * (c[3].y - c[3].x), -s * (c[3].x + c[3].y));   // * e^{-3 i pi/4}
    Dft<R, 4>::run(b);
    Dft<R, 4>::run(c);
#pragma unroll
    for (int m = 0; m < 4; m++) {
      v[2 * m] = b[m];
      v[2 * m + 1] = c[m];
    }
  }
};

// Asynchronous global -> shared copy of one element (cp.async): a thread issues
// all of its loads of a tile without waiting for any of them.
template <class T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src),
               "n"((int)sizeof(T))
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__host__ __device__ constexpr int first_radix(int n) {
  int p = 1;
  while (p * 8 <= n) p *= 8;
  return (n / p == 1) ? 8 : n / p;
}

// One Stockham pass of radix RAD over NFFT transforms of length n held in buf:
// element e of transform f lives at buf[f * FS + e * ES].  Butterfly j reads
// e = j + t n/RAD, multiplies by w^{(j mod NS) t n/(NS RAD)} (w = e^{-2 pi i/n})
// and writes e = (j / NS) NS RAD + (j mod NS) + t NS.  tw[k] = e^{-2 pi i k/(n TWS)}.
// With PAD > 0 logical slot i is stored at i + (i >> PAD) (one gap every 2^PAD
// elements), which spreads the strided writes of the first passes over the banks.
template <int PAD> __device__ __forceinline__ int padded(int i) { return PAD ? i + (i >> PAD) : i; }

template <class R, int n, int RAD, int NS, int NFFT, int NT, int FS, int ES, bool FFAST, int TWS, int PAD>
__device__ __forceinline__ void fft_pass(cx<R>* buf, const cx<R>* __restrict__ tw) {
  constexpr int NBF = n / RAD;
  constexpr int NB = NFFT * NBF;
  constexpr int BPT = (NB + NT - 1) / NT;
  cx<R> v[BPT][RAD];
#pragma unroll
  for (int i = 0; i < BPT; i++) {
    const int b = threadIdx.x + i * NT;
    if ((NB % NT) == 0 || b < NB) {
      const int f = FFAST ? (b % NFFT) : (b / NBF);
      const int j = FFAST ? (b / NFFT) : (b % NBF);
      const int jm = j & (NS - 1);
      // twiddles w^t, t < RAD; radix 8 loads w, w^2, w^4 and forms the other
      // four by products (three table reads instead of seven)
      cx<R> w[RAD];
      if constexpr (NS > 1) {
        const int s1 = jm * (n / (NS * RAD)) * TWS;
        if constexpr (RAD == 8) {
          w[1] = tw[s1];
          w[2] = tw[2 * s1];
          w[4] = tw[4 * s1];
          w[3] = cmul<R>(w[1], w[2]);
          w[5] = cmul<R>(w[4], w[1]);
          w[6] = cmul<R>(w[4], w[2]);
          w[7] = cmul<R>(w[4], w[3]);
        } else {
#pragma unroll
          for (int t = 1; t < RAD; t++) w[t] = tw[t * s1];
        }
      }
#pragma unroll
      for (int t = 0; t < RAD; t++) {
        cx<R> a = buf[padded<PAD>(f * FS + (j + t * NBF) * ES)];
        if (NS > 1 && t > 0) a = cmul<R>(a, w[t]);
        v[i][t] = a;
      }
      Dft<R, RAD>::run(v[i]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < BPT; i++) {
    const int b = threadIdx.x + i * NT;
    if ((NB % NT) == 0 || b < NB) {
      const int f = FFAST ? (b % NFFT) : (b / NBF);
      const int j = FFAST ? (b / NFFT) : (b % NBF);
      const int jm = j & (NS - 1);
      const int base = (j / NS) * NS * RAD + jm;
#pragma unroll
      for (int t = 0; t < RAD; t++) buf[padded<PAD>(f * FS + (base + t * NS) * ES)] = v[i][t];
    }
  }
  __syncthreads();
}

template <class R, int n, int NS, int NFFT, int NT, int FS, int ES, bool FFAST, int TWS, int PAD = 0>
__device__ __forceinline__ void fft_all(cx<R>* buf, const cx<R>* __restrict__ tw) {
  if constexpr (NS < n) {
    constexpr int RAD = (NS == 1) ? first_radix(n) : 8;
    fft_pass<R, n, RAD, NS, NFFT, NT, FS, ES, FFAST, TWS, PAD>(buf, tw);
    fft_all<R, n, NS * RAD, NFFT, NT, FS, ES, FFAST, TWS, PAD>(buf, tw);
  }
}

constexpr int FFT_NT = 256;

// Rows per CTA of the row kernels, and columns per CTA strip of the column kernel,
// chosen so that one CTA holds 2048 (rows) or 8192 / 4096 (columns) complex values.
template <class R, int N> struct RowCfg {
  static constexpr int ROWS = (2048 / (N / 2)) > 0 ? 2048 / (N / 2) : 1;
  static constexpr int PAD = 4;                                   // see padded()
  static constexpr int SLOTS = ROWS * (N / 2) + ((ROWS * (N / 2)) >> PAD);
};
template <class R, int N> struct ColCfg {
  static constexpr int ELEMS = sizeof(R) == 4 ? 8192 : 4096;
  static constexpr int SW0 = ELEMS / N;
  static constexpr int SW = SW0 < 1 ? 1 : (SW0 > N / 2 ? N / 2 : SW0);
};

// ---------------------------------------------------------------------------
// rows_fwd: real rows of length N -> packed half spectrum rows (N/2 complex).
// ---------------------------------------------------------------------------
// PADIN: the rows are those of an N/2 x N/2 image per band, zero-padded to
// N x N (input pitch N/2, upper half of each row zero; rows = (N/2) L); output
// row r of band l goes to row l N + r (rows N/2..N-1 of each band are not written).
template <class R, int N, bool PADIN = false>
__global__ void __launch_bounds__(FFT_NT) k_rows_fwd(const R* __restrict__ in, cx<R>* __restrict__ out,
                                                     int rows, const cx<R>* __restrict__ tw) {
  constexpr int n = N / 2;
  constexpr int ROWS = RowCfg<R, N>::ROWS;
  constexpr int PAD = RowCfg<R, N>::PAD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R>* buf = reinterpret_cast<cx<R>*>(smem_raw);
  const int row0 = blockIdx.x * ROWS;
  const cx<R>* src = reinterpret_cast<const cx<R>*>(in);
  for (int e = threadIdx.x; e < ROWS * n; e += FFT_NT) {
    const int r = e / n, m = e % n;
    if (row0 + r < rows && (!PADIN || m < n / 2))
      cp_async_elem(buf + padded<PAD>(e), src + (size_t)(row0 + r) * (PADIN ? n / 2 : n) + m);
    else buf[padded<PAD>(e)] = mk<R>(0, 0);
  }
  cp_async_wait_all();
  __syncthreads();
  fft_all<R, n, 1, ROWS, FFT_NT, n, 1, false, 2, PAD>(buf, tw);
  for (int e = threadIdx.x; e < ROWS * n; e += FFT_NT) {
    const int r = e / n, k = e % n;
    if (row0 + r >= rows) continue;
    const size_t orow = PADIN ? (size_t)((row0 + r) / (N / 2)) * N + (row0 + r) % (N / 2) : (size_t)(row0 + r);
    const cx<R> Zk = buf[padded<PAD>(r * n + k)];
    cx<R> P;
    if (k == 0) {
      P = mk<R>(Zk.x + Zk.y, Zk.x - Zk.y);  // (X[0], X[N/2]), both real
    } else {
      const cx<R> Zm = cconj<R>(buf[padded<PAD>(r * n + (n - k))]);
      const cx<R> E = cscale<R>(cadd<R>(Zk, Zm), (R)0.5);
      const cx<R> D = csub<R>(Zk, Zm);
      const cx<R> O = mk<R>((R)0.5 * D.y, (R)-0.5 * D.x);  // D / (2i)
      P = cadd<R>(E, cmul<R>(tw[k], O));
    }
    out[orow * n + k] = P;
  }
}

// ---------------------------------------------------------------------------
// rows_inv: packed half spectrum rows -> real rows (times N).
// ---------------------------------------------------------------------------
// CROP: only rows 0..N/2-1 of each band (rows = (N/2) L; row r of band l read
// from row l N + r) and only their first N/2 values, written with pitch N/2.
template <class R, int N, bool CROP = false>
__global__ void __launch_bounds__(FFT_NT) k_rows_inv(const cx<R>* __restrict__ in, R* __restrict__ out,
                                                     int rows, const cx<R>* __restrict__ tw) {
  constexpr int n = N / 2;
  constexpr int ROWS = RowCfg<R, N>::ROWS;
  constexpr int PAD = RowCfg<R, N>::PAD;
  constexpr int EPT = (ROWS * n + FFT_NT - 1) / FFT_NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R>* buf = reinterpret_cast<cx<R>*>(smem_raw);
  const int row0 = blockIdx.x * ROWS;
  for (int e = threadIdx.x; e < ROWS * n; e += FFT_NT) {
    const int r = e / n, m = e % n;
    const size_t irow = CROP ? (size_t)((row0 + r) / (N / 2)) * N + (row0 + r) % (N / 2) : (size_t)(row0 + r);
    if (row0 + r < rows) cp_async_elem(buf + padded<PAD>(e), in + irow * n + m);
    else buf[padded<PAD>(e)] = mk<R>(0, 0);
  }
  cp_async_wait_all();
  __syncthreads();
  cx<R> z[EPT];
#pragma unroll
  for (int i = 0; i < EPT; i++) {
    const int e = threadIdx.x + i * FFT_NT;
    if (e < ROWS * n) {
      const int r = e / n, k = e % n;
      cx<R> Z;
      if (k == 0) {
        const cx<R> P = buf[padded<PAD>(r * n)];
        Z = mk<R>(P.x + P.y, P.x - P.y);  // E' + i O' with E' = X0 + Xn, O' = X0 - Xn
      } else {
        const cx<R> Xk = buf[padded<PAD>(r * n + k)];
        const cx<R> Xm = cconj<R>(buf[padded<PAD>(r * n + (n - k))]);
        const cx<R> E = cadd<R>(Xk, Xm);
        const cx<R> O = cmul<R>(csub<R>(Xk, Xm), cconj<R>(tw[k]));
        Z = mk<R>(E.x - O.y, E.y + O.x);  // E + i O
      }
      z[i] = cconj<R>(Z);  // inverse through the forward transform of the conjugate
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < EPT; i++) {
    const int e = threadIdx.x + i * FFT_NT;
    if (e < ROWS * n) buf[padded<PAD>(e)] = z[i];
  }
  __syncthreads();
  fft_all<R, n, 1, ROWS, FFT_NT, n, 1, false, 2, PAD>(buf, tw);
  cx<R>* dst = reinterpret_cast<cx<R>*>(out);
  for (int e = threadIdx.x; e < ROWS * n; e += FFT_NT) {
    const int r = e / n, m = e % n;
    if (row0 + r >= rows || (CROP && m >= n / 2)) continue;
    const cx<R> y = buf[padded<PAD>(e)];
    dst[(size_t)(row0 + r) * (CROP ? n / 2 : n) + m] = mk<R>(y.x, -y.y);  // x[2m] = Re conj(y), x[2m+1] = Im conj(y)
  }
}

// ---------------------------------------------------------------------------
// cols: strip of SW packed columns of one band, COLS_NT threads (two
// butterflies per thread and pass at N = 1024, so the operands of a pass stay
// in few registers).
// ---------------------------------------------------------------------------
// MODE 1: X = c + g B, then the inverse column transform (conjugate trick).
// MODE 2 is MODE 1 plus the data-fit partials 1/2 ||y - H x||^2 (Parseval over the
// half spectrum: interior columns count twice) read from hh/yh.
// MODE 3 applies H (X = h B) and MODE 4 applies Q^-1 alone (X = g B): both serve
// the backward pass.  MODE 5 applies H^T (X = conj(h) B), for the conjugate
// gradient step I of a linear convolution.
// The filter is applied in place in shared memory.  Packed column 0 holds the
// DC column (A) and the Nyquist column (B) as A + iB; unpacking row ky needs
// row (N - ky) mod N, so one thread takes both rows of a mirror pair.
constexpr int COLS_NT = 512;

template <class R, int MODE>
struct ColFilter {
  const cx<R>* cc;
  const R* gg;
  const cx<R>* hh;
  const cx<R>* yh;
  // X^ of one bin from B^ = Z; MODE 2 adds wfit |F(y) - N^2 h X^|^2 to fit
  __device__ __forceinline__ cx<R> apply(cx<R> Z, size_t o, R N2, R& fit, R wfit) const {
    cx<R> Xh;
    if (MODE == 3) Xh = cscale<R>(cmul<R>(hh[o], Z), (R)1 / N2);
    else if (MODE == 5) Xh = cscale<R>(cmul<R>(cconj<R>(hh[o]), Z), (R)1 / N2);
    else if (MODE == 4) Xh = cscale<R>(Z, gg[o]);
    else Xh = cadd<R>(cc[o], cscale<R>(Z, gg[o]));
    if (MODE == 2) {
      const cx<R> r = csub<R>(yh[o], cscale<R>(cmul<R>(hh[o], Xh), N2));
      fit = fma(wfit, r.x * r.x + r.y * r.y, fit);
    }
    return Xh;
  }
};

// PRUNE (MODE 3 / 5): the spatial rows N/2..N-1 of the input are zero (they
// are not read) and only the output rows 0..N/2-1 are written (a zero-padded
// image in, its [0, N/2) rows out).
template <class R, int N, int MODE, bool PRUNE = false>
__global__ void __launch_bounds__(COLS_NT, 2) k_cols(cx<R>* __restrict__ work, const cx<R>* __restrict__ tw,
                                                  cx<R>* __restrict__ out_main, cx<R>* __restrict__ out_nyq,
                                                  const cx<R>* __restrict__ cc, const cx<R>* __restrict__ cc_nyq,
                                                  const R* __restrict__ gg, const R* __restrict__ gg_nyq,
                                                  const cx<R>* __restrict__ hh, const cx<R>* __restrict__ hh_nyq,
                                                  const cx<R>* __restrict__ yh, const cx<R>* __restrict__ yh_nyq,
                                                  double* __restrict__ partials) {
  constexpr int n = N / 2;          // packed columns per band
  constexpr int SW = ColCfg<R, N>::SW;
  constexpr int EL = N * SW;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<R>* buf = reinterpret_cast<cx<R>*>(smem_raw);
  const int strips = n / SW;
  const int band = blockIdx.x / strips;
  const int kx0 = (blockIdx.x % strips) * SW;
  cx<R>* base = work + (size_t)band * N * n + kx0;
  for (int e = threadIdx.x; e < EL; e += COLS_NT) {
    const int ky = e / SW, c = e % SW;
    if (PRUNE && ky >= N / 2) buf[e] = mk<R>(0, 0);
    else cp_async_elem(buf + e, base + (size_t)ky * n + c);
  }
  if (MODE != 0) {
    // L2 prefetch of the strip's filter constants (read after the forward
    // transform): one line per row of the strip and array
    const size_t b0 = (size_t)band * N * n + kx0;
    for (int ky = threadIdx.x; ky < N; ky += COLS_NT) {
      const size_t o = b0 + (size_t)ky * n;
      if (MODE == 1 || MODE == 2) {
        asm volatile("prefetch.global.L2 [%0];" ::"l"(cc + o));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(gg + o));
      }
      if (MODE == 4) asm volatile("prefetch.global.L2 [%0];" ::"l"(gg + o));
      if (MODE == 2 || MODE == 3 || MODE == 5) asm volatile("prefetch.global.L2 [%0];" ::"l"(hh + o));
      if (MODE == 2) asm volatile("prefetch.global.L2 [%0];" ::"l"(yh + o));
    }
  }
  cp_async_wait_all();
  __syncthreads();
  fft_all<R, N, 1, SW, COLS_NT, 1, SW, true, 1>(buf, tw);

  if constexpr (MODE == 0) {
    // forward transform only: unpacked spectrum out
    for (int e = threadIdx.x; e < EL; e += COLS_NT) {
      const int ky = e / SW, c = e % SW, kx = kx0 + c;
      const cx<R> Z = buf[e];
      const size_t o = ((size_t)band * N + ky) * n + kx;
      if (kx == 0) {
        const cx<R> Zm = cconj<R>(buf[((N - ky) % N) * SW]);
        const cx<R> A = cscale<R>(cadd<R>(Z, Zm), (R)0.5);
        const cx<R> D = csub<R>(Z, Zm);
        const cx<R> B = mk<R>((R)0.5 * D.y, (R)-0.5 * D.x);
        out_main[o] = A;
        out_nyq[(size_t)band * N + ky] = B;
      } else {
        out_main[o] = Z;
      }
    }
  } else {
    const R N2 = (R)N * (R)N;
    const ColFilter<R, MODE> fm{cc, gg, hh, yh};
    const ColFilter<R, MODE> fn{cc_nyq, gg_nyq, hh_nyq, yh_nyq};
    R fit = 0;  // this thread's 16 or so bins in the cube's precision; FP64 from the block sum on
    auto unpack_row = [&](int ky, cx<R> Z, cx<R> Zmir) {
      // row ky of column 0 from Z = buf[ky] and Zmir = buf[(N - ky) mod N]
      const cx<R> Zm = cconj<R>(Zmir);
      const cx<R> A = cscale<R>(cadd<R>(Z, Zm), (R)0.5);
      const cx<R> D = csub<R>(Z, Zm);
      const cx<R> B = mk<R>((R)0.5 * D.y, (R)-0.5 * D.x);
      const size_t o = ((size_t)band * N + ky) * n, on = (size_t)band * N + ky;
      const cx<R> Ax = fm.apply(A, o, N2, fit, (R)1), Bx = fn.apply(B, on, N2, fit, (R)1);
      return cconj<R>(mk<R>(Ax.x - Bx.y, Ax.y + Bx.x));  // conj(A' + i B')
    };
#pragma unroll 4
    for (int e = threadIdx.x; e < EL; e += COLS_NT) {
      const int ky = e / SW, c = e % SW, kx = kx0 + c;
      if (kx == 0) {
        if (ky > N / 2) continue;  // the partner of a pair with ky < N/2
        const int km = (N - ky) & (N - 1);
        const cx<R> Z = buf[ky * SW], Zp = buf[km * SW];
        const cx<R> v = unpack_row(ky, Z, Zp);
        if (km != ky) buf[km * SW] = unpack_row(km, Zp, Z);
        buf[ky * SW] = v;
      } else {
        const size_t o = ((size_t)band * N + ky) * n + kx;
        buf[e] = cconj<R>(fm.apply(buf[e], o, N2, fit, (R)2));
      }
    }
    __syncthreads();
    fft_all<R, N, 1, SW, COLS_NT, 1, SW, true, 1>(buf, tw);
    for (int e = threadIdx.x; e < EL; e += COLS_NT) {
      const int ky = e / SW, c = e % SW;
      if (PRUNE && ky >= N / 2) continue;
      base[(size_t)ky * n + c] = cconj<R>(buf[e]);
    }
    if (MODE == 2) {
      // in the cube's precision: FP32 plans take the FP32 warp stage of the reduction
      R q[Q_COUNT];
#pragma unroll
      for (int i = 0; i < Q_COUNT; i++) q[i] = 0;
      q[Q_XMIN] = (R)1e300;  // infinite in FP32; the reduction writes the FP64 sentinel
      q[Q_FIT] = fit * (R)(0.5 / ((double)N * (double)N));
      block_reduce_write<COLS_NT>(q, partials + (size_t)blockIdx.x * MF_NQ);
    }
  }
}

// ---------------------------------------------------------------------------
// g = 1/((|h|^2 + rho) N^2),  c = conj(h) yhat g
// ---------------------------------------------------------------------------
template <class R>
__global__ void k_constants(const cx<R>* __restrict__ hh, const cx<R>* __restrict__ yh, cx<R>* __restrict__ cc,
                            R* __restrict__ gg, size_t count, R rho, R invN2) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const cx<R> h = hh[i], y = yh[i];
    const R g = invN2 / (h.x * h.x + h.y * h.y + rho);
    gg[i] = g;
    cc[i] = mk<R>((h.x * y.x + h.y * y.y) * g, (h.x * y.y - h.y * y.x) * g);
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <class R, int N>
static cudaError_t rows_fwd_n(const R* in, cx<R>* out, int rows, const cx<R>* tw, cudaStream_t s) {
  constexpr int ROWS = RowCfg<R, N>::ROWS;
  const size_t sm = sizeof(cx<R>) * RowCfg<R, N>::SLOTS;
  cudaError_t e = cudaFuncSetAttribute(k_rows_fwd<R, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_rows_fwd<R, N><<<(rows + ROWS - 1) / ROWS, FFT_NT, sm, s>>>(in, out, rows, tw);
  return cudaGetLastError();
}
template <class R, int N>
static cudaError_t rows_inv_n(const cx<R>* in, R* out, int rows, const cx<R>* tw, cudaStream_t s) {
  constexpr int ROWS = RowCfg<R, N>::ROWS;
  const size_t sm = sizeof(cx<R>) * RowCfg<R, N>::SLOTS;
  cudaError_t e = cudaFuncSetAttribute(k_rows_inv<R, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_rows_inv<R, N><<<(rows + ROWS - 1) / ROWS, FFT_NT, sm, s>>>(in, out, rows, tw);
  return cudaGetLastError();
}
template <class R, int N, int MODE>
static cudaError_t cols_mode(cx<R>* work, int L, const cx<R>* tw, cx<R>* om, cx<R>* on, const cx<R>* cc,
                             const cx<R>* ccn, const R* gg, const R* ggn, const cx<R>* hh, const cx<R>* hhn,
                             const cx<R>* yh, const cx<R>* yhn, double* partials, cudaStream_t s) {
  constexpr int SW = ColCfg<R, N>::SW;
  const size_t sm = sizeof(cx<R>) * N * SW;
  const int blocks = L * ((N / 2) / SW);
  cudaError_t e = cudaFuncSetAttribute(k_cols<R, N, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_cols<R, N, MODE><<<blocks, COLS_NT, sm, s>>>(work, tw, om, on, cc, ccn, gg, ggn, hh, hhn, yh, yhn, partials);
  return cudaGetLastError();
}
template <class R, int N>
static cudaError_t cols_n(cx<R>* work, int L, const cx<R>* tw, int mode, cx<R>* om, cx<R>* on, const cx<R>* cc,
                          const cx<R>* ccn, const R* gg, const R* ggn, const cx<R>* hh, const cx<R>* hhn,
                          const cx<R>* yh, const cx<R>* yhn, double* partials, cudaStream_t s) {
  if (mode == 0) return cols_mode<R, N, 0>(work, L, tw, om, on, cc, ccn, gg, ggn, hh, hhn, yh, yhn, partials, s);
  if (mode == 1) return cols_mode<R, N, 1>(work, L, tw, om, on, cc, ccn, gg, ggn, hh, hhn, yh, yhn, partials, s);
  if (mode == 3) return cols_mode<R, N, 3>(work, L, tw, om, on, cc, ccn, gg, ggn, hh, hhn, yh, yhn, partials, s);
  if (mode == 4) return cols_mode<R, N, 4>(work, L, tw, om, on, cc, ccn, gg, ggn, hh, hhn, yh, yhn, partials, s);
  if (mode == 5) return cols_mode<R, N, 5>(work, L, tw, om, on, cc, ccn, gg, ggn, hh, hhn, yh, yhn, partials, s);
  return cols_mode<R, N, 2>(work, L, tw, om, on, cc, ccn, gg, ggn, hh, hhn, yh, yhn, partials, s);
}

template <class R, int N, bool PADIN>
static cudaError_t rows_fwd_v(const R* in, cx<R>* out, int rows, const cx<R>* tw, cudaStream_t s) {
  constexpr int ROWS = RowCfg<R, N>::ROWS;
  const size_t sm = sizeof(cx<R>) * RowCfg<R, N>::SLOTS;
  cudaError_t e = cudaFuncSetAttribute(k_rows_fwd<R, N, PADIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_rows_fwd<R, N, PADIN><<<(rows + ROWS - 1) / ROWS, FFT_NT, sm, s>>>(in, out, rows, tw);
  return cudaGetLastError();
}
template <class R, int N, bool CROP>
static cudaError_t rows_inv_v(const cx<R>* in, R* out, int rows, const cx<R>* tw, cudaStream_t s) {
  constexpr int ROWS = RowCfg<R, N>::ROWS;
  const size_t sm = sizeof(cx<R>) * RowCfg<R, N>::SLOTS;
  cudaError_t e = cudaFuncSetAttribute(k_rows_inv<R, N, CROP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_rows_inv<R, N, CROP><<<(rows + ROWS - 1) / ROWS, FFT_NT, sm, s>>>(in, out, rows, tw);
  return cudaGetLastError();
}
template <class R, int N, int MODE>
static cudaError_t cols_pruned_v(cx<R>* work, int L, const cx<R>* tw, const cx<R>* hh, const cx<R>* hhn,
                                 cudaStream_t s) {
  constexpr int SW = ColCfg<R, N>::SW;
  const size_t sm = sizeof(cx<R>) * N * SW;
  const int blocks = L * ((N / 2) / SW);
  cudaError_t e =
      cudaFuncSetAttribute(k_cols<R, N, MODE, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_cols<R, N, MODE, true><<<blocks, COLS_NT, sm, s>>>(work, tw, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                       nullptr, hh, hhn, nullptr, nullptr, nullptr);
  return cudaGetLastError();
}

template <class R>
int cols_blocks(int N, int L) {
  const int sw0 = (sizeof(R) == 4 ? 8192 : 4096) / N;
  const int sw = sw0 < 1 ? 1 : (sw0 > N / 2 ? N / 2 : sw0);
  return L * ((N / 2) / sw);
}

#define MF_SWITCH_N(N, CALL)          \
  switch (N) {                        \
    case 16: return CALL(16);         \
    case 32: return CALL(32);         \
    case 64: return CALL(64);         \
    case 128: return CALL(128);       \
    case 256: return CALL(256);       \
    case 512: return CALL(512);       \
    case 1024: return CALL(1024);     \
    case 2048: return CALL(2048);     \
    default: return cudaErrorInvalidValue; \
  }

template <class R>
cudaError_t launch_rows_fwd(const R* in, cx<R>* out, int N, int rows, const cx<R>* tw, cudaStream_t s) {
#define CALL(NN) rows_fwd_n<R, NN>(in, out, rows, tw, s)
  MF_SWITCH_N(N, CALL)
#undef CALL
}
template <class R>
cudaError_t launch_rows_inv(const cx<R>* in, R* out, int N, int rows, const cx<R>* tw, cudaStream_t s) {
#define CALL(NN) rows_inv_n<R, NN>(in, out, rows, tw, s)
  MF_SWITCH_N(N, CALL)
#undef CALL
}
template <class R>
cudaError_t launch_cols(cx<R>* work, int N, int L, const cx<R>* tw, int mode, cx<R>* out_main, cx<R>* out_nyq,
                        const cx<R>* cc, const cx<R>* cc_nyq, const R* gg, const R* gg_nyq, const cx<R>* hh,
                        const cx<R>* hh_nyq, const cx<R>* yh, const cx<R>* yh_nyq, double* partials,
                        cudaStream_t s) {
#define CALL(NN) \
  cols_n<R, NN>(work, L, tw, mode, out_main, out_nyq, cc, cc_nyq, gg, gg_nyq, hh, hh_nyq, yh, yh_nyq, partials, s)
  MF_SWITCH_N(N, CALL)
#undef CALL
}

template <class R>
cudaError_t launch_constants(const cx<R>* hh, const cx<R>* hh_nyq, const cx<R>* yh, const cx<R>* yh_nyq,
                             cx<R>* cc, cx<R>* cc_nyq, R* gg, R* gg_nyq, int N, int L, double rho_bar,
                             cudaStream_t s) {
  const R invN2 = (R)(1.0 / ((double)N * (double)N));
  const size_t cm = (size_t)L * N * (N / 2), cn = (size_t)L * N;
  k_constants<R><<<(unsigned)((cm + 255) / 256 < 65535 * 8 ? (cm + 255) / 256 : 65535 * 8), 256, 0, s>>>(
      hh, yh, cc, gg, cm, (R)rho_bar, invN2);
  k_constants<R><<<(unsigned)((cn + 255) / 256), 256, 0, s>>>(hh_nyq, yh_nyq, cc_nyq, gg_nyq, cn, (R)rho_bar, invN2);
  return cudaGetLastError();
}

// The zero-padded 2-D convolution of an (M/2) x (M/2) image through M x M
// transforms that skip what is known to be zero or not needed (FP32): rows of
// the padded image in, the column pass on the first M/2 spatial rows, the
// [0, M/2)^2 region out (see the PADIN, PRUNE and CROP variants above).
#define MF_SWITCH_M(M, CALL)          \
  switch (M) {                        \
    case 32: return CALL(32);         \
    case 64: return CALL(64);         \
    case 128: return CALL(128);       \
    case 256: return CALL(256);       \
    case 512: return CALL(512);       \
    case 1024: return CALL(1024);     \
    case 2048: return CALL(2048);     \
    default: return cudaErrorInvalidValue; \
  }

cudaError_t launch_rows_fwd_pad(const float* in, cx<float>* out, int M, int rows, const cx<float>* tw,
                                cudaStream_t s) {
#define CALL(MM) rows_fwd_v<float, MM, true>(in, out, rows, tw, s)
  MF_SWITCH_M(M, CALL)
#undef CALL
}
cudaError_t launch_rows_inv_crop(const cx<float>* in, float* out, int M, int rows, const cx<float>* tw,
                                 cudaStream_t s) {
#define CALL(MM) rows_inv_v<float, MM, true>(in, out, rows, tw, s)
  MF_SWITCH_M(M, CALL)
#undef CALL
}
cudaError_t launch_cols_pruned(cx<float>* work, int M, int L, const cx<float>* tw, int mode, const cx<float>* hh,
                               const cx<float>* hh_nyq, cudaStream_t s) {
  if (mode == 3) {
#define CALL(MM) cols_pruned_v<float, MM, 3>(work, L, tw, hh, hh_nyq, s)
    MF_SWITCH_M(M, CALL)
#undef CALL
  }
  if (mode == 5) {
#define CALL(MM) cols_pruned_v<float, MM, 5>(work, L, tw, hh, hh_nyq, s)
    MF_SWITCH_M(M, CALL)
#undef CALL
  }
  return cudaErrorInvalidValue;
}

#define INST(R)                                                                                          \
  template cudaError_t launch_rows_fwd<R>(const R*, cx<R>*, int, int, const cx<R>*, cudaStream_t);       \
  template cudaError_t launch_rows_inv<R>(const cx<R>*, R*, int, int, const cx<R>*, cudaStream_t);       \
  template cudaError_t launch_cols<R>(cx<R>*, int, int, const cx<R>*, int, cx<R>*, cx<R>*, const cx<R>*, \
                                      const cx<R>*, const R*, const R*, const cx<R>*, const cx<R>*,      \
                                      const cx<R>*, const cx<R>*, double*, cudaStream_t);                \
  template int cols_blocks<R>(int, int);                                                                 \
  template cudaError_t launch_constants<R>(const cx<R>*, const cx<R>*, const cx<R>*, const cx<R>*, cx<R>*, \
                                           cx<R>*, R*, R*, int, int, double, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace mf
