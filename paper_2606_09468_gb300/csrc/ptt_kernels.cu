// Device code of the FP64 pseudo-spectral sPTT channel step (2D, sm_103a).
//
// One step (Sec. 2: fully dealiased Fourier-Chebyshev pseudo-spectral method,
// fourth-order semi-implicit BDF) is the launch sequence
//   k_ycols  (inverse)  spectral (m, n) -> values on the padded Gauss-Lobatto
//                       y grid, with d/dy by the Chebyshev recurrence
//   k_xfused            per padded y row: inverse x FFTs of 14 fields, the
//                       sPTT / advection products of Eqs. 1-2, forward x FFTs
//   k_ycols  (forward)  padded y values -> Chebyshev coefficients (truncated)
//   k_spec              per Fourier mode, out of shared memory: linear
//                       explicit terms, curl-curl forcing, SBDF sums, the
//                       quasi-tridiagonal tau solves, u from continuity
//   k_tick              step counters
// followed by the diagnostics of Sec. 3 (k_ycols x2, k_xrows, k_diag_part,
// k_diag_count, k_diag_mid, k_diag_final).  All transforms are mixed-radix (2, 3, 4, 5) Stockham FFTs
// in shared memory; the Chebyshev transforms are discrete cosine transforms
// of type I computed as FFTs of the even extension.
//
// Layouts: spectral arrays [member][field][m][n] (each mode's Chebyshev
// column contiguous); values on a y grid [member][field][j][m] (each y row's
// Fourier modes contiguous).
#include <cstdio>

#include "ptt_internal.h"

namespace ptt {
namespace {

// ------------------------------------------------------------ complex math
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscl(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 mul_i(double2 a) { return make_double2(-a.y, a.x); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cfma(double s, double2 a, double2 c) {  // s*a + c
  return make_double2(fma(s, a.x, c.x), fma(s, a.y, c.y));
}
__device__ __forceinline__ double2 czero() { return make_double2(0.0, 0.0); }

// single precision twins (mixed-precision transforms)
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscl(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 mul_i(float2 a) { return make_float2(-a.y, a.x); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cfma(float s, float2 a, float2 c) {
  return make_float2(fmaf(s, a.x, c.x), fmaf(s, a.y, c.y));
}

template <typename C2> struct RealOf;
template <> struct RealOf<double2> { using T = double; };
template <> struct RealOf<float2> { using T = float; };
template <typename C2> __device__ __forceinline__ C2 zero2();
template <> __device__ __forceinline__ double2 zero2<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 zero2<float2>() { return make_float2(0.f, 0.f); }
template <typename D> __device__ __forceinline__ D cvt2(double2 v);
template <typename D> __device__ __forceinline__ D cvt2(float2 v);
template <> __device__ __forceinline__ double2 cvt2<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 cvt2<float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }
template <> __device__ __forceinline__ double2 cvt2<double2>(float2 v) { return make_double2(v.x, v.y); }
template <> __device__ __forceinline__ float2 cvt2<float2>(float2 v) { return v; }

// ------------------------------------------------------------ radix DFTs
// DIR = -1: exp(-2 pi i jk/R) (forward); DIR = +1: exp(+2 pi i jk/R).
template <int DIR, int R> struct Bfly;

template <int DIR> struct Bfly<DIR, 2> {
  template <typename C2>
  static __device__ __forceinline__ void run(C2* v) {
    C2 t = v[0];
    v[0] = cadd(t, v[1]);
    v[1] = csub(t, v[1]);
  }
};

template <int DIR> struct Bfly<DIR, 4> {
  template <typename C2>
  static __device__ __forceinline__ void run(C2* v) {
    C2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    C2 s13 = cadd(v[1], v[3]), d13 = mul_i(csub(v[1], v[3]));
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    if (DIR < 0) { v[1] = csub(d02, d13); v[3] = cadd(d02, d13); }
    else         { v[1] = cadd(d02, d13); v[3] = csub(d02, d13); }
  }
};

template <int DIR> struct Bfly<DIR, 3> {
  template <typename C2>
  static __device__ __forceinline__ void run(C2* v) {
    using T = typename RealOf<C2>::T;
    const T s = (T)(DIR * 0.86602540378443864676);  // sin(2 pi / 3), signed
    C2 t1 = cadd(v[1], v[2]);
    C2 it2 = mul_i(csub(v[1], v[2]));
    C2 m = cfma((T)-0.5, t1, v[0]);
    v[0] = cadd(v[0], t1);
    v[1] = cfma(s, it2, m);
    v[2] = cfma(-s, it2, m);
  }
};

template <int DIR> struct Bfly<DIR, 5> {
  template <typename C2>
  static __device__ __forceinline__ void run(C2* v) {
    using T = typename RealOf<C2>::T;
    const T c1 = (T)0.30901699437494742410;   // cos(2 pi / 5)
    const T c2 = (T)-0.80901699437494742410;  // cos(4 pi / 5)
    const T s1 = (T)(DIR * 0.95105651629515357212);  // sin(2 pi / 5), signed
    const T s2 = (T)(DIR * 0.58778525229247312917);  // sin(4 pi / 5), signed
    C2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    C2 t3 = mul_i(csub(v[1], v[4])), t4 = mul_i(csub(v[2], v[3]));
    C2 b1 = cfma(c1, t1, cfma(c2, t2, v[0]));
    C2 b2 = cfma(c2, t1, cfma(c1, t2, v[0]));
    C2 e1 = cfma(s1, t3, cscl(t4, s2));
    C2 e2 = cfma(s2, t3, cscl(t4, -s1));
    v[0] = cadd(v[0], cadd(t1, t2));
    v[1] = cadd(b1, e1);
    v[4] = csub(b1, e1);
    v[2] = cadd(b2, e2);
    v[3] = csub(b2, e2);
  }
};

// One Stockham pass of radix R over nl lines (line l at offset l*ls).
template <int DIR, int R, typename C2>
__device__ __forceinline__ void fft_pass(const C2* __restrict__ src, C2* __restrict__ dst,
                                         int nl, int ls, int n, int Ns,
                                         const C2* __restrict__ tw) {
  const int nb = n / R;
  const int st = n / (Ns * R);
  const int total = nl * nb;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int l = t / nb;
    const int j = t - l * nb;
    const C2* s = src + l * ls;
    C2* d = dst + l * ls;
    const int jm = j % Ns;
    C2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = s[j + r * nb];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C2 w = __ldg(&tw[jm * r * st]);
        if (DIR > 0) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    Bfly<DIR, R>::run(v);
    const int o = (j / Ns) * Ns * R + jm;
#pragma unroll
    for (int r = 0; r < R; ++r) d[o + r * Ns] = v[r];
  }
}

template <typename C2> __device__ __forceinline__ const C2* plan_tw(const FftPlan& pl);
template <> __device__ __forceinline__ const double2* plan_tw<double2>(const FftPlan& pl) { return pl.tw; }
template <> __device__ __forceinline__ const float2* plan_tw<float2>(const FftPlan& pl) { return pl.twf; }

// Unnormalised DFT of nl lines of length pl.n held in `a`, using `b` as the
// ping-pong buffer.  Returns the buffer holding the result.  Must be called
// by the whole block after a __syncthreads(); ends with one.
template <int DIR, typename C2>
__device__ C2* fft_lines(C2* a, C2* b, int nl, int ls, const FftPlan& pl) {
  C2* src = a;
  C2* dst = b;
  const C2* tw = plan_tw<C2>(pl);
  int Ns = 1;
  for (int s = 0; s < pl.nst; ++s) {
    const int R = pl.radix[s];
    switch (R) {
      case 2: fft_pass<DIR, 2>(src, dst, nl, ls, pl.n, Ns, tw); break;
      case 3: fft_pass<DIR, 3>(src, dst, nl, ls, pl.n, Ns, tw); break;
      case 4: fft_pass<DIR, 4>(src, dst, nl, ls, pl.n, Ns, tw); break;
      default: fft_pass<DIR, 5>(src, dst, nl, ls, pl.n, Ns, tw); break;
    }
    __syncthreads();
    Ns *= R;
    C2* t = src; src = dst; dst = t;
  }
  return src;
}

// SBDF coefficients, orders 1..4: a_0..a_4 and b_0..b_3 (Sec. 2: 4th-order
// semi-implicit BDF; lower orders start the history).
__constant__ double c_sa[4][5] = {{1.0, -1.0, 0.0, 0.0, 0.0},
                                  {1.5, -2.0, 0.5, 0.0, 0.0},
                                  {11.0 / 6.0, -3.0, 1.5, -1.0 / 3.0, 0.0},
                                  {25.0 / 12.0, -4.0, 3.0, -4.0 / 3.0, 0.25}};
__constant__ double c_sb[4][4] = {{1.0, 0.0, 0.0, 0.0},
                                  {2.0, -1.0, 0.0, 0.0},
                                  {3.0, -3.0, 1.0, 0.0},
                                  {4.0, -6.0, 4.0, -1.0}};

// ------------------------------------------- warp-cooperative recurrences
// FP64 runs at a few lanes per clock per SM on this part, so a warp FP64
// instruction costs the same pipe time whether 1 or 32 lanes are active.
// The Chebyshev recurrences and the tau sweeps are therefore written as
// warp scans: each lane takes a contiguous chunk, composes it sequentially,
// and the chunks are combined with shuffles.
constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxChunk = 8;  // tau sweeps: up to 8 rows per lane (ny <= 513)

__device__ __forceinline__ double2 shfl_down2(double2 v, int o) {
  return make_double2(__shfl_down_sync(kFull, v.x, o), __shfl_down_sync(kFull, v.y, o));
}
__device__ __forceinline__ float2 shfl_down2(float2 v, int o) {
  return make_float2(__shfl_down_sync(kFull, v.x, o), __shfl_down_sync(kFull, v.y, o));
}
__device__ __forceinline__ double2 shfl_up2(double2 v, int o) {
  return make_double2(__shfl_up_sync(kFull, v.x, o), __shfl_up_sync(kFull, v.y, o));
}
__device__ __forceinline__ double2 warp_allsum2(double2 v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(kFull, v.x, o);
    v.y += __shfl_xor_sync(kFull, v.y, o);
  }
  return v;
}

// Chebyshev derivative by one warp: out_n = (2/c_n) sum_{p > n, p + n odd} p a_p
// (c_0 = 2), as two same-parity suffix sums T(k) = sum_{p >= k, p = k mod 2} p a_p
// with out_{k-1} = (2/c_{k-1}) T(k).  `out` must not alias `a`.
template <typename C2>
__device__ void warp_cheb_deriv(const C2* a, C2* out, int N) {
  using T = typename RealOf<C2>::T;
  const int lane = threadIdx.x & 31;
  for (int par = 0; par < 2; ++par) {
    const int L = (N - par + 1) / 2;
    const int c = (L + 31) / 32;
    const int i0 = min(lane * c, L), i1 = min(i0 + c, L);
    C2 acc = zero2<C2>();
    for (int i = i1 - 1; i >= i0; --i) {
      const int k = par + 2 * i;
      acc = cfma((T)k, a[k], acc);
      if (k >= 1) out[k - 1] = cscl(acc, (T)(k == 1 ? 1 : 2));
    }
    C2 inc = acc;
    for (int o = 1; o < 32; o <<= 1) {
      const C2 v = shfl_down2(inc, o);
      if (lane + o < 32) inc = cadd(inc, v);
    }
    C2 ex = shfl_down2(inc, 1);
    if (lane == 31) ex = zero2<C2>();
    for (int i = i0; i < i1; ++i) {
      const int k = par + 2 * i;
      if (k >= 1) out[k - 1] = cfma((T)(k == 1 ? 1 : 2), ex, out[k - 1]);
    }
  }
  if (lane == 0) out[N - 1] = zero2<C2>();
  __syncwarp();
}

// Warp-cooperative quasi-tridiagonal tau solve (system stated at k_spec): the backward
// elimination P_i = alpha_i + beta_i P_{i+1} and the forward substitution
// a_i = P_i + Q_i a_{i-1} are affine recurrences, evaluated as warp scans of
// affine maps; the boundary sums are warp reductions.  `out` may alias R.
__device__ void warp_qt_solve(int N, int p, double alpha, const double2* R, double2* out,
                              const double* Q, const double* inv, const double* F, double G,
                              const double* w1, const double* w2, const double* w3,
                              double bcfac, double rsign) {
  const int lane = threadIdx.x & 31;
  const int L = (N - p + 1) / 2;  // unknowns a_{p+2i}, i < L; rows i = 1..L-1
  const int nr = L - 1;
  const int c = (nr + 31) / 32;
  const int i0 = min(1 + lane * c, L), i1 = min(i0 + c, L);
  double2 al[kMaxChunk];
  double be[kMaxChunk];
  double2 rs = czero();
#pragma unroll
  for (int t = 0; t < kMaxChunk; ++t) {
    const int i = i0 + t;
    if (t < c && i < i1) {
      const int n = p + 2 * i;
      const double2 Rm2 = cscl(R[n - 2], rsign);
      const double2 R0 = cscl(R[n], rsign);
      const double cc = (n == 2) ? 2.0 : 1.0;
      double2 r = cscl(Rm2, -cc * w1[n]);
      if (n <= N - 3) r = cfma(w2[n], R0, r);
      double un = 0.0;
      if (n <= N - 5) {
        r = cfma(-w3[n], cscl(R[n + 2], rsign), r);
        un = -alpha * w3[n];
      }
      al[t] = cscl(r, inv[n]);
      be[t] = -un * inv[n];
      rs = cadd(rs, R0);
    } else {
      al[t] = czero();
      be[t] = 1.0;
    }
  }
  if (lane == 0) rs = cadd(rs, cscl(R[p], rsign));
  __syncwarp();
  // backward: chunk map P_{i0} = A + B P_{i1}
  double2 A = czero();
  double B = 1.0;
#pragma unroll
  for (int t = kMaxChunk - 1; t >= 0; --t) {
    if (t < c && i0 + t < i1) {
      A = cfma(be[t], A, al[t]);
      B *= be[t];
    }
  }
  double2 SA = A;
  double SB = B;
  for (int o = 1; o < 32; o <<= 1) {
    const double2 hA = shfl_down2(SA, o);
    const double hB = __shfl_down_sync(kFull, SB, o);
    if (lane + o < 32) {
      SA = cfma(SB, hA, SA);
      SB *= hB;
    }
  }
  double2 Pin = shfl_down2(SA, 1);
  if (lane == 31) Pin = czero();
  double2 U = czero();
  double2 P = Pin;
#pragma unroll
  for (int t = kMaxChunk - 1; t >= 0; --t) {
    const int i = i0 + t;
    if (t < c && i < i1) {
      const int n = p + 2 * i;
      P = cfma(be[t], P, al[t]);
      out[n] = P;
      U = cfma(F[n], P, U);
    }
  }
  U = warp_allsum2(U);
  rs = warp_allsum2(rs);
  const double2 a0 = cscl(csub(cscl(rs, bcfac), U), G);
  // forward: chunk map a_{i1-1} = C + D a_{i0-1}
  double2 Cc = czero();
  double Dd = 1.0;
  double2 Pv[kMaxChunk];
  double Qv[kMaxChunk];
#pragma unroll
  for (int t = 0; t < kMaxChunk; ++t) {
    const int i = i0 + t;
    if (t < c && i < i1) {
      const int n = p + 2 * i;
      Pv[t] = out[n];
      Qv[t] = Q[n];
      Cc = cfma(Qv[t], Cc, Pv[t]);
      Dd *= Qv[t];
    }
  }
  double2 IC = Cc;
  double ID = Dd;
  for (int o = 1; o < 32; o <<= 1) {
    const double2 hC = shfl_up2(IC, o);
    const double hD = __shfl_up_sync(kFull, ID, o);
    if (lane >= o) {
      IC = cfma(ID, hC, IC);
      ID *= hD;
    }
  }
  double2 EC = shfl_up2(IC, 1);
  double ED = __shfl_up_sync(kFull, ID, 1);
  if (lane == 0) { EC = czero(); ED = 1.0; }
  double2 av = cfma(ED, a0, EC);
  __syncwarp();
#pragma unroll
  for (int t = 0; t < kMaxChunk; ++t) {
    const int i = i0 + t;
    if (t < c && i < i1) {
      av = cfma(Qv[t], av, Pv[t]);
      out[p + 2 * i] = av;
    }
  }
  if (lane == 0) out[p] = a0;
  __syncwarp();
}

// ---------------------------------------------- per-mode spectral stage
// ------------------------------------------------------ Chebyshev columns
// Column transforms along y for a batch of members and fields.  Coefficient
// side: column m, row n at m*cm + n*cn; value side: column m, row j at
// m*vm + j*vj (within one field of one member).  Input and output may be in
// double or single precision independently of the compute type.
struct YJob {
  const void* src;
  void* dst;
  long long src_mstride, dst_mstride;  // per member (elements)
  long long src_fstride, dst_fstride;  // per field (elements)
  int src_field[8];
  int src_field2[8];  // inverse only: >= 0 adds this field to src_field
  int dst_field[8];
  int deriv[8];       // inverse only: transform d/dy of the field
  long long cm, cn;   // coefficient-side strides
  long long vm, vj;   // value-side strides
  int K;              // columns
  int N, M;           // Chebyshev modes, grid intervals / points
  int inverse;        // 1: coefficients -> values; 0: values -> coefficients (N rows)
  int gauss;          // 0: M+1 Gauss-Lobatto points (DCT-I, FFT length 2M);
                      // 1: M Gauss points (DCT-II/III, FFT length M, M even)
  int src_f32, dst_f32;  // element types of src / dst (0: complex double, 1: complex float)
  const double2* tw4;    // gauss: tw4[k] = exp(-i pi k / (2M)), k < M
  const float2* tw4f;    // the same in single precision
  int C;              // columns per block
  const int* status;  // skip members with status != 0 (may be null)
  FftPlan pl;
};

template <typename CT>
__device__ __forceinline__ CT ld2(const void* p, long long i, int f32) {
  return f32 ? cvt2<CT>(static_cast<const float2*>(p)[i]) : cvt2<CT>(static_cast<const double2*>(p)[i]);
}
template <typename CT>
__device__ __forceinline__ void st2(void* p, long long i, int f32, CT v) {
  if (f32) static_cast<float2*>(p)[i] = cvt2<float2>(v);
  else static_cast<double2*>(p)[i] = cvt2<double2>(v);
}
template <typename CT> __device__ __forceinline__ CT ld_tw4(const YJob& J, int k);
template <> __device__ __forceinline__ double2 ld_tw4<double2>(const YJob& J, int k) { return __ldg(&J.tw4[k]); }
template <> __device__ __forceinline__ float2 ld_tw4<float2>(const YJob& J, int k) { return __ldg(&J.tw4f[k]); }

// Values at the M Gauss points y_j = cos(pi (2j+1)/(2M)) from coefficients
// (DCT-III) and back (DCT-II), each as one complex FFT of length M: the
// output (input) order is permuted v_n = f_{2n}, v_{M-1-n} = f_{2n+1}, and a
// quarter-period twiddle exp(-+ i pi k/(2M)) maps between the two (Makhoul's
// construction; the real and imaginary parts of a column ride in one FFT).
template <typename CT>
__device__ void ycols_gauss(const YJob& J, const void* src, const void* src2, void* dst,
                            CT* A, CT* B, int c0, int nc) {
  using T = typename RealOf<CT>::T;
  const int C = J.C, N = J.N, Mg = J.M;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int f = blockIdx.y;
  if (J.inverse) {
    for (int i = tid; i < Mg * C; i += nt) {
      const int c = i / Mg, n = i - c * Mg;
      CT v = zero2<CT>();
      if (c < nc && n < N) {
        const long long o = (c0 + c) * J.cm + n * J.cn;
        v = ld2<CT>(src, o, J.src_f32);
        if (src2) v = cadd(v, ld2<CT>(src2, o, J.src_f32));
      }
      A[i] = v;
    }
    __syncthreads();
    if (J.deriv[f]) {
      for (int c = tid >> 5; c < C; c += (nt >> 5)) warp_cheb_deriv(A + c * Mg, B + c * Mg, N);
      __syncthreads();
      for (int i = tid; i < N * C; i += nt) {
        const int c = i / N, n = i - c * N;
        A[c * Mg + n] = B[c * Mg + n];
      }
      __syncthreads();
    }
    // V_0 = a_0, V_k = (1/2) exp(+i pi k/(2M)) (a_k - i a_{M-k})
    for (int i = tid; i < Mg * C; i += nt) {
      const int c = i / Mg, k = i - c * Mg;
      const CT ak = A[i];
      CT V;
      if (k == 0) {
        V = ak;
      } else {
        const CT amk = A[c * Mg + Mg - k];
        const CT w = cconj(ld_tw4<CT>(J, k));
        V = cscl(cmul(w, csub(ak, mul_i(amk))), (T)0.5);
      }
      B[i] = V;
    }
    __syncthreads();
    CT* res = fft_lines<+1>(B, A, C, Mg, J.pl);
    for (int i = tid; i < Mg * C; i += nt) {
      const int j = i / C, c = i - j * C;
      if (c < nc) {
        const int pos = (j & 1) ? (Mg - 1 - (j >> 1)) : (j >> 1);
        st2<CT>(dst, j * J.vj + (c0 + c) * J.vm, J.dst_f32, res[c * Mg + pos]);
      }
    }
  } else {
    for (int i = tid; i < Mg * C; i += nt) {
      const int j = i / C, c = i - j * C;
      const int pos = (j & 1) ? (Mg - 1 - (j >> 1)) : (j >> 1);
      A[c * Mg + pos] = (c < nc) ? ld2<CT>(src, j * J.vj + (c0 + c) * J.vm, J.src_f32) : zero2<CT>();
    }
    __syncthreads();
    CT* res = fft_lines<-1>(A, B, C, Mg, J.pl);
    const T s0 = (T)(1.0 / Mg), s1 = (T)(2.0 / Mg);
    for (int i = tid; i < N * C; i += nt) {
      const int c = i / N, k = i - c * N;
      if (c < nc) {
        const CT Vk = res[c * Mg + k];
        const CT Vm = cconj(res[c * Mg + (k == 0 ? 0 : Mg - k)]);
        const CT Vr = cscl(cadd(Vk, Vm), (T)0.5);
        const CT d = csub(Vk, Vm);
        CT Vi;
        Vi.x = (T)0.5 * d.y;
        Vi.y = (T)-0.5 * d.x;
        const CT w = ld_tw4<CT>(J, k);
        const T xr = w.x * Vr.x - w.y * Vr.y;
        const T xi = w.x * Vi.x - w.y * Vi.y;
        const T sc = (k == 0) ? s0 : s1;
        CT o;
        o.x = sc * xr;
        o.y = sc * xi;
        st2<CT>(dst, (c0 + c) * J.cm + k * J.cn, J.dst_f32, o);
      }
    }
  }
}

// Gauss-Lobatto path (double precision only): DCT-I by the even extension.
__device__ void ycols_lobatto(const YJob& J, const void* srcv, const void* src2v, void* dstv,
                              double2* A, double2* B, double2* a0s, int c0, int nc) {
  const int C = J.C, N = J.N, M = J.M, P = 2 * J.M;
  const double2* src = static_cast<const double2*>(srcv);
  const double2* src2 = static_cast<const double2*>(src2v);
  double2* dst = static_cast<double2*>(dstv);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int f = blockIdx.y;
  if (J.inverse) {
    for (int i = tid; i < N * C; i += nt) {
      const int c = i / N, n = i - c * N;
      double2 v = czero();
      if (c < nc) {
        const long long o = (c0 + c) * J.cm + n * J.cn;
        v = src[o];
        if (src2) v = cadd(v, src2[o]);
      }
      A[c * P + n] = v;
    }
    __syncthreads();
    if (J.deriv[f]) {
      for (int c = tid >> 5; c < C; c += (nt >> 5)) warp_cheb_deriv(A + c * P, B + c * P, N);
      __syncthreads();
      for (int i = tid; i < N * C; i += nt) {
        const int c = i / N, n = i - c * N;
        A[c * P + n] = B[c * P + n];
      }
      __syncthreads();
    }
    if (tid < C) {
      a0s[tid] = A[tid * P];
      a0s[C + tid] = (N > M) ? A[tid * P + M] : czero();
    }
    // even extension: A[n] = a_n (n <= M, zero for n >= N), A[P-n] = a_n
    for (int i = tid; i < C * P; i += nt) {
      const int c = i / P, n = i - c * P;
      if (n >= N && n <= M) A[i] = czero();
      else if (n > M) { const int r = P - n; A[i] = (r < N) ? A[c * P + r] : czero(); }
    }
    __syncthreads();
    double2* res = fft_lines<-1>(A, B, C, P, J.pl);
    // f_j = (F_j + a_0 + (-1)^j a_M) / 2
    for (int i = tid; i < (M + 1) * C; i += nt) {
      const int j = i / C, c = i - j * C;
      if (c < nc) {
        double2 v = cadd(res[c * P + j], a0s[c]);
        v = (j & 1) ? csub(v, a0s[C + c]) : cadd(v, a0s[C + c]);
        dst[j * J.vj + (c0 + c) * J.vm] = cscl(v, 0.5);
      }
    }
  } else {
    for (int i = tid; i < (M + 1) * C; i += nt) {
      const int j = i / C, c = i - j * C;
      A[c * P + j] = (c < nc) ? src[j * J.vj + (c0 + c) * J.vm] : czero();
    }
    __syncthreads();
    for (int i = tid; i < C * P; i += nt) {
      const int c = i / P, j = i - c * P;
      if (j > M) A[i] = A[c * P + (P - j)];
    }
    __syncthreads();
    double2* res = fft_lines<-1>(A, B, C, P, J.pl);
    const double inv = 1.0 / M;
    for (int i = tid; i < N * C; i += nt) {
      const int c = i / N, n = i - c * N;
      if (c < nc) {
        const double s = (n == 0 || n == M) ? 0.5 * inv : inv;
        dst[(c0 + c) * J.cm + n * J.cn] = cscl(res[c * P + n], s);
      }
    }
  }
}

template <typename CT>
__global__ void __launch_bounds__(256) k_ycols(YJob J) {
  const int b = blockIdx.z;
  if (J.status && J.status[b]) return;
  const int f = blockIdx.y;
  // FFT length per column: M on the Gauss grid, 2M (even extension) on the
  // Gauss-Lobatto grid; shared memory holds 2 C lines of it (+ 2 C scalars)
  const int C = J.C, K = J.K, P = J.gauss ? J.M : 2 * J.M;
  const int c0 = blockIdx.x * C;
  const int nc = min(C, K - c0);
  extern __shared__ __align__(16) unsigned char smraw[];
  CT* A = reinterpret_cast<CT*>(smraw);
  CT* B = A + (size_t)C * P;
  const size_t es = J.src_f32 ? sizeof(float2) : sizeof(double2);
  const size_t ed = J.dst_f32 ? sizeof(float2) : sizeof(double2);
  const void* src = static_cast<const char*>(J.src) + (b * J.src_mstride + J.src_field[f] * J.src_fstride) * es;
  void* dst = static_cast<char*>(J.dst) + (b * J.dst_mstride + J.dst_field[f] * J.dst_fstride) * ed;
  const void* src2 = (J.inverse && J.src_field2[f] >= 0)
      ? static_cast<const char*>(J.src) + (b * J.src_mstride + J.src_field2[f] * J.src_fstride) * es
      : nullptr;
  if (J.gauss) {
    ycols_gauss<CT>(J, src, src2, dst, A, B, c0, nc);
  } else if constexpr (sizeof(CT) == sizeof(double2)) {
    ycols_lobatto(J, src, src2, dst, reinterpret_cast<double2*>(A), reinterpret_cast<double2*>(B),
                  reinterpret_cast<double2*>(B) + (size_t)C * P, c0, nc);
  }
}

// ---------------------------------------------------------- Fourier rows
// Row transforms along x: complex modes m < K <-> real values at n points,
// two real fields packed in one complex line.
struct XJob {
  const double2* srcC;  // c2r: complex rows
  const double* srcR;   // r2c: real rows
  double2* dstC;
  double* dstR;
  long long src_mstride, dst_mstride, src_fstride, dst_fstride;
  int src_rstep, dst_rstep;  // row index multipliers (elements per row = K or n)
  int nf;                    // fields (<= 6)
  int K, n;
  int c2r;
  const int* status;
  FftPlan pl;
};

__global__ void __launch_bounds__(256) k_xrows(XJob J) {
  const int b = blockIdx.y;
  if (J.status && J.status[b]) return;
  const int row = blockIdx.x;
  const int K = J.K, n = J.n, nf = J.nf, nl = (nf + 1) / 2;
  extern __shared__ double2 sm[];
  double2* A = sm;
  double2* Bb = sm + (size_t)nl * n;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (J.c2r) {
    const double2* src = J.srcC + b * J.src_mstride + (long long)row * J.src_rstep * K;
    for (int i = tid; i < nl * n; i += nt) {
      const int l = i / n, k = i - l * n;
      const int fa = 2 * l, fb = 2 * l + 1;
      int kk = -1;
      bool cj = false;
      if (k < K) kk = k;
      else if (k > n - K) { kk = n - k; cj = true; }
      double2 h = czero();
      if (kk >= 0) {
        double2 F = src[fa * J.src_fstride + kk];
        double2 G = (fb < nf) ? src[fb * J.src_fstride + kk] : czero();
        if (kk == 0) { F.y = 0.0; G.y = 0.0; }
        if (cj) { F = cconj(F); G = cconj(G); }
        h = cadd(F, mul_i(G));
      }
      A[i] = h;
    }
    __syncthreads();
    double2* res = fft_lines<+1>(A, Bb, nl, n, J.pl);
    double* dst = J.dstR + b * J.dst_mstride + (long long)row * J.dst_rstep * n;
    for (int i = tid; i < nl * n; i += nt) {
      const int l = i / n, x = i - l * n;
      const double2 h = res[i];
      dst[(2 * l) * J.dst_fstride + x] = h.x;
      if (2 * l + 1 < nf) dst[(2 * l + 1) * J.dst_fstride + x] = h.y;
    }
  } else {
    const double* src = J.srcR + b * J.src_mstride + (long long)row * J.src_rstep * n;
    for (int i = tid; i < nl * n; i += nt) {
      const int l = i / n, x = i - l * n;
      const double fa = src[(2 * l) * J.src_fstride + x];
      const double fb = (2 * l + 1 < nf) ? src[(2 * l + 1) * J.src_fstride + x] : 0.0;
      A[i] = make_double2(fa, fb);
    }
    __syncthreads();
    double2* res = fft_lines<-1>(A, Bb, nl, n, J.pl);
    double2* dst = J.dstC + b * J.dst_mstride + (long long)row * J.dst_rstep * K;
    const double inv = 1.0 / n;
    for (int i = tid; i < nl * K; i += nt) {
      const int l = i / K, k = i - l * K;
      const double2 hk = res[l * n + k];
      const double2 hm = cconj(res[l * n + (k == 0 ? 0 : n - k)]);
      // F = (hk + conj(h_{-k}))/2, G = (hk - conj(h_{-k}))/(2i)
      const double2 F = cscl(cadd(hk, hm), 0.5 * inv);
      const double2 d = csub(hk, hm);
      const double2 G = make_double2(0.5 * inv * d.y, -0.5 * inv * d.x);
      dst[(2 * l) * J.dst_fstride + k] = F;
      if (2 * l + 1 < nf) dst[(2 * l + 1) * J.dst_fstride + k] = G;
    }
  }
}

// ------------------------------------------------ fused x pass + products
// Yp fields: 0 u, 1 v, 2 du/dy, 3 cxx, 4 cxy, 5 cyy, 6 dcxx/dy, 7 dcxy/dy, 8 dcyy/dy.
// Physical lines (pairs re/im): (u, v) (uy, ux) (vx, cxx) (cxy, cyy)
// (cxx_y, cxy_y) (cyy_y, cxx_x) (cxy_x, cyy_x).
__constant__ int c_xsrc[14] = {0, 1, 2, 0, 1, 3, 4, 5, 6, 7, 8, 3, 4, 5};
__constant__ int c_xik[14] = {0, 0, 0, 1, 1, 0, 0, 0, 0, 0, 0, 1, 1, 1};

template <typename C2> __device__ __forceinline__ const C2* yp_ptr(const GroupDev& g);
template <> __device__ __forceinline__ const double2* yp_ptr<double2>(const GroupDev& g) { return g.Yp; }
template <> __device__ __forceinline__ const float2* yp_ptr<float2>(const GroupDev& g) { return g.Ypf; }
template <typename C2> __device__ __forceinline__ C2* zp_ptr(const GroupDev& g);
template <> __device__ __forceinline__ double2* zp_ptr<double2>(const GroupDev& g) { return g.Zp; }
template <> __device__ __forceinline__ float2* zp_ptr<float2>(const GroupDev& g) { return g.Zpf; }

// C2 = double2: the FP64 path; C2 = float2: the mixed path (FP32 transforms
// and products, FP64 state and solves).
template <typename C2>
__global__ void __launch_bounds__(512) k_xfused(GroupDev g) {
  using T = typename RealOf<C2>::T;
  const int b = blockIdx.y;
  if (g.status[b]) return;
  const int j = blockIdx.x;
  const int K = g.K, Mx = g.Mx, rows = g.M;
  const MemberPrm pr = g.prm[b];
  extern __shared__ __align__(16) unsigned char smraw[];
  C2* A = reinterpret_cast<C2*>(smraw);
  C2* B = A + 7 * Mx;
  const C2* Y = yp_ptr<C2>(g) + (size_t)b * 9 * rows * K + (size_t)j * K;
  const T kfac = (T)(2.0 * 3.14159265358979323846 / pr.lx);
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < 7 * Mx; i += nt) {
    const int l = i / Mx, k = i - l * Mx;
    int kk = -1;
    bool cj = false;
    if (k < K) kk = k;
    else if (k > Mx - K) { kk = Mx - k; cj = true; }
    C2 h = zero2<C2>();
    if (kk >= 0) {
      const int fa = 2 * l, fb = 2 * l + 1;
      C2 F = Y[(size_t)c_xsrc[fa] * rows * K + kk];
      C2 G = Y[(size_t)c_xsrc[fb] * rows * K + kk];
      if (kk == 0) { F.y = 0; G.y = 0; }
      const T km = kfac * kk;
      if (c_xik[fa]) F = cscl(mul_i(F), km);
      if (c_xik[fb]) G = cscl(mul_i(G), km);
      if (cj) { F = cconj(F); G = cconj(G); }
      h = cadd(F, mul_i(G));
    }
    A[i] = h;
  }
  __syncthreads();
  C2* res = fft_lines<+1>(A, B, 7, Mx, g.plMx);
  C2* oth = (res == A) ? B : A;
  const T eps = (T)pr.eps, iwi = (T)pr.inv_wi;
  for (int x = tid; x < Mx; x += nt) {
    const C2 h0 = res[x], h1 = res[Mx + x], h2 = res[2 * Mx + x], h3 = res[3 * Mx + x];
    const C2 h4 = res[4 * Mx + x], h5 = res[5 * Mx + x], h6 = res[6 * Mx + x];
    const T u = h0.x, v = h0.y, uy = h1.x, ux = h1.y, vx = h2.x, cxx = h2.y;
    const T cxy = h3.x, cyy = h3.y, cxx_y = h4.x, cxy_y = h4.y, cyy_y = h5.x;
    const T cxx_x = h5.y, cxy_x = h6.x, cyy_x = h6.y;
    // Eq. 1: L_ij = du_i/dx_j (L_yy = -ux by continuity); relaxation factor
    // f = 1 + eps Tr(c - I) with c_zz = 1.
    const T rw = ((T)1 + eps * (cxx + cyy - (T)2)) * iwi;
    const T ncxx = -(u * cxx_x + v * cxx_y) + (T)2 * (ux * cxx + uy * cxy) - (cxx - (T)1) * rw;
    const T ncxy = -(u * cxy_x + v * cxy_y) + uy * cyy + vx * cxx - cxy * rw;
    const T ncyy = -(u * cyy_x + v * cyy_y) + (T)2 * (vx * cxy - ux * cyy) - (cyy - (T)1) * rw;
    // Eq. 2 advection
    const T nu_ = -(u * ux + v * uy);
    const T nv_ = -(u * vx - v * ux);
    C2 o0, o1, o2;
    o0.x = ncxx; o0.y = ncxy;
    o1.x = ncyy; o1.y = nu_;
    o2.x = nv_; o2.y = 0;
    oth[x] = o0;
    oth[Mx + x] = o1;
    oth[2 * Mx + x] = o2;
  }
  __syncthreads();
  C2* r2 = fft_lines<-1>(oth, res, 3, Mx, g.plMx);
  C2* Z = zp_ptr<C2>(g) + (size_t)b * 5 * rows * K + (size_t)j * K;
  const T inv = (T)(1.0 / Mx);
  for (int i = tid; i < 3 * K; i += nt) {
    const int l = i / K, k = i - l * K;
    const C2 hk = r2[l * Mx + k];
    const C2 hm = cconj(r2[l * Mx + (k == 0 ? 0 : Mx - k)]);
    const C2 F = cscl(cadd(hk, hm), (T)0.5 * inv);
    const C2 d = csub(hk, hm);
    C2 G;
    G.x = (T)0.5 * inv * d.y;
    G.y = (T)-0.5 * inv * d.x;
    Z[(size_t)(2 * l) * rows * K + k] = F;
    if (l < 2) Z[(size_t)(2 * l + 1) * rows * K + k] = G;
  }
}

// The tau system solved per (mode, system, parity) by warp_qt_solve:
//   (alpha - beta D^2) a = rsign * R   on tau rows n <= N-3,
//   sum_{n = p mod 2} a_n = bcfac * sum_{n = p mod 2} rsign * R_n,
// taken in the three-term form that integrating twice gives (rows n >= 2);
// beta enters only through the operator tables.

// One block per (member, Fourier mode m).  Every column of the mode lives in
// shared memory; the recurrences (Chebyshev derivatives, tau sweeps) run as
// warp scans, the rest in parallel over the Chebyshev index.  256 threads:
// the eight (system, parity) solves get a warp each.
//   explicit terms (Eq. 2): H_x = N_u + gam (i k c_xx + D c_xy) (+ 2/Re on the
//     mean mode), H_y = N_v + gam (i k c_xy + D c_yy); forcing of the evolved
//     velocity quantity: -D(i k H_x) - k^2 H_y (m >= 1, phi = lap v), H_x (m = 0)
//   evolved quantities x = (c_xx, c_xy, c_yy, q), q = (D^2 - k^2) v or U
//   SBDF sums R = sum_j (-a_{j+1}/dt) x^{n-j} + b_j N^{n-j} (Sec. 2: 4th-order
//     semi-implicit BDF, orders 1-3 on the first steps)
//   tau solves: c with the wall rows of Eq. 1 at kappa = 0; velocity by
//     phi-Helmholtz, v-Poisson and the influence correction v'(+-1) = 0
//   u = i (D v) / k from continuity (Eq. 3)
// mode 1: only H_x, H_y into Rb[0], Rb[1] (explicit right-hand side).
__global__ void __launch_bounds__(256) k_spec(GroupDev g, int mode) {
  const int b = blockIdx.y;
  const int m = blockIdx.x;
  if (g.status[b]) return;
  const int K = g.K, N = g.N, nb = g.nb;
  const size_t NK = (size_t)N * K;
  const MemberPrm pr = g.prm[b];
  const long long cnt = g.count[b];
  const int slot = (int)(cnt & 3);
  const int o = (cnt < 3) ? (int)cnt : 3;
  const double km = 2.0 * 3.14159265358979323846 * m / pr.lx;
  const double km2 = km * km;
  extern __shared__ double2 sm[];
  double2* sc0 = sm;            // c_xx  -> new c_xx
  double2* sc1 = sm + N;        // c_xy  -> new c_xy
  double2* sc2 = sm + 2 * N;    // c_yy  -> new c_yy
  double2* sv = sm + 3 * N;     // v     -> new v
  double2* shx = sm + 4 * N;    // N_u   -> H_x
  double2* shy = sm + 5 * N;    // N_v   -> H_y -> new u
  double2* sq = sm + 6 * N;     // q
  double2* snq = sm + 7 * N;    // forcing of q
  double2* sR = sm + 8 * N;     // R[4][N]
  double* tb = reinterpret_cast<double*>(sm + 12 * N);  // [3 sys][Q, inv, F][N], vh[N]
  const double2* X = g.X + (size_t)b * 5 * NK + (size_t)m * N;
  const double2* NR = g.NR + (size_t)b * 5 * NK + (size_t)m * N;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < N; i += nt) {
    sc0[i] = X[2 * NK + i];
    sc1[i] = X[3 * NK + i];
    sc2[i] = X[4 * NK + i];
    sv[i] = X[NK + i];
    shx[i] = NR[3 * NK + i];
    shy[i] = NR[4 * NK + i];
    if (m == 0) sq[i] = X[i];
  }
  if (mode == 0) {
    const double* qt = g.qt + ((size_t)b * 4 + o) * 3 * 3 * NK + (size_t)m * N;
    for (int i = tid; i < 9 * N; i += nt) {
      const int w = i / N, n = i - w * N;
      tb[i] = qt[(size_t)w * NK + n];
    }
    const double* vh = g.vh + ((size_t)b * 4 + o) * NK + (size_t)m * N;
    for (int i = tid; i < N; i += nt) tb[9 * N + i] = vh[i];
  }
  __syncthreads();
  // derivatives, one warp each: D c_xy -> sR[0], D c_yy -> sR[1], D v -> sR[2] -> D^2 v -> sq
  {
    const int warp = tid >> 5;
    if (warp == 0) warp_cheb_deriv(sc1, sR, N);
    else if (warp == 1) warp_cheb_deriv(sc2, sR + N, N);
    else if (warp == 2 && mode == 0 && m != 0) {
      warp_cheb_deriv(sv, sR + 2 * N, N);
      warp_cheb_deriv(sR + 2 * N, sq, N);
    }
  }
  __syncthreads();
  for (int n = tid; n < N; n += nt) {
    double2 hx = cadd(shx[n], cscl(cadd(cscl(mul_i(sc0[n]), km), sR[n]), pr.gam));
    const double2 hy = cadd(shy[n], cscl(cadd(cscl(mul_i(sc1[n]), km), sR[N + n]), pr.gam));
    if (m == 0 && n == 0) hx.x += pr.forcing;
    shx[n] = hx;
    shy[n] = hy;
    if (mode == 0 && m != 0) sq[n] = cfma(-km2, sv[n], sq[n]);
  }
  __syncthreads();
  if (mode == 1) {
    double2* R = g.Rb + (size_t)b * 4 * NK + (size_t)m * N;
    for (int i = tid; i < N; i += nt) {
      R[i] = shx[i];
      R[NK + i] = shy[i];
    }
    return;
  }
  // forcing of q: m >= 1: -D(i k H_x) - k^2 H_y; m = 0: H_x
  if (m != 0 && tid < 32) warp_cheb_deriv(shx, sR, N);
  __syncthreads();
  for (int n = tid; n < N; n += nt)
    snq[n] = (m == 0) ? shx[n] : csub(cscl(mul_i(sR[n]), -km), cscl(shy[n], km2));
  __syncthreads();
  // history slot and SBDF sums
  {
    double2* E = g.Eh + ((size_t)slot * nb + b) * 4 * NK + (size_t)m * N;
    double2* Nn = g.Nh + ((size_t)slot * nb + b) * 4 * NK + (size_t)m * N;
    const double idt = 1.0 / pr.dt;
    for (int i = tid; i < N; i += nt) {
      const double2 x[4] = {sc0[i], sc1[i], sc2[i], sq[i]};
      const double2 nn[4] = {NR[i], NR[NK + i], NR[2 * NK + i], snq[i]};
      double2 acc[4];
      for (int s = 0; s < 4; ++s) {
        E[s * NK + i] = x[s];
        Nn[s * NK + i] = nn[s];
        acc[s] = cfma(c_sb[o][0], nn[s], cscl(x[s], -c_sa[o][1] * idt));
      }
      for (int jj = 1; jj <= o; ++jj) {
        const size_t sl = (size_t)((slot - jj) & 3);
        const double2* Eo = g.Eh + (sl * nb + b) * 4 * NK + (size_t)m * N + i;
        const double2* No = g.Nh + (sl * nb + b) * 4 * NK + (size_t)m * N + i;
        const double ca = -c_sa[o][jj + 1] * idt, cb = c_sb[o][jj];
        for (int s = 0; s < 4; ++s) acc[s] = cfma(cb, No[s * NK], cfma(ca, Eo[s * NK], acc[s]));
      }
      for (int s = 0; s < 4; ++s) sR[s * N + i] = acc[s];
    }
  }
  __syncthreads();
  const double* w1 = g.wrow;
  const double* w2 = g.wrow + N;
  const double* w3 = g.wrow + 2 * N;
  const double a0 = c_sa[o][0];
  {  // eight (system, parity) tau solves, one warp each
    const int t = tid >> 5;
    const int sys = t >> 1, p = t & 1;
    auto G = [&](int ts) { return g.qtG[((((size_t)b * 4 + o) * 3 + ts) * 2 + p) * K + m]; };
    const double* T0 = tb;
    const double* T1 = tb + 3 * N;
    const double* T2 = tb + 6 * N;
    const int lane = tid & 31;
    if (sys < 3) {
      double2* out = sm + (size_t)sys * N;  // sc0, sc1, sc2
      const double2* R = sR + (size_t)sys * N;
      const double alpha = a0 / pr.dt + pr.kappa * km2;
      if (pr.kappa == 0.0) {
        const double ia = 1.0 / alpha;
        for (int n = p + 2 * lane; n < N; n += 64) out[n] = cscl(R[n], ia);
      } else {
        warp_qt_solve(N, p, alpha, R, out, T0, T0 + N, T0 + 2 * N, G(0), w1, w2, w3, pr.dt / a0,
                      1.0);
      }
    } else if (m == 0) {
      warp_qt_solve(N, p, a0 / pr.dt, sR + 3 * N, shy, T1, T1 + N, T1 + 2 * N, G(1), w1, w2, w3,
                    0.0, 1.0);
      for (int n = p + 2 * lane; n < N; n += 64) sv[n] = czero();
    } else {
      double2* Rv = sR + 3 * N;
      warp_qt_solve(N, p, a0 / pr.dt + pr.nu * km2, Rv, Rv, T1, T1 + N, T1 + 2 * N, G(1), w1, w2,
                    w3, 0.0, 1.0);
      warp_qt_solve(N, p, km2, Rv, sv, T2, T2 + N, T2 + 2 * N, G(2), w1, w2, w3, 0.0, -1.0);
      double2 sacc = czero();
      for (int n = p + 2 * lane; n < N; n += 64) sacc = cfma((double)n * n, sv[n], sacc);
      sacc = warp_allsum2(sacc);
      const double* vh = tb + 9 * N;
      const double2 coef = cscl(sacc, -g.vhS[(((size_t)b * 4 + o) * 2 + p) * K + m]);
      for (int n = p + 2 * lane; n < N; n += 64)
        sv[n] = make_double2(fma(coef.x, vh[n], sv[n].x), fma(coef.y, vh[n], sv[n].y));
    }
  }
  __syncthreads();
  // u = i (D v) / k (m >= 1), continuity
  if (m != 0) {
    if (tid < 32) warp_cheb_deriv(sv, sR, N);
    __syncthreads();
    const double ik = 1.0 / km;
    for (int n = tid; n < N; n += nt) shy[n] = cscl(mul_i(sR[n]), ik);
    __syncthreads();
  }
  double2* Xw = g.X + (size_t)b * 5 * NK + (size_t)m * N;
  for (int i = tid; i < N; i += nt) {
    Xw[i] = shy[i];
    Xw[NK + i] = sv[i];
    Xw[2 * NK + i] = sc0[i];
    Xw[3 * NK + i] = sc1[i];
    Xw[4 * NK + i] = sc2[i];
  }
}

// Advance the step counters (after every block of k_spec has read them).
__global__ void k_tick(GroupDev g) {
  const int b = threadIdx.x + blockIdx.x * blockDim.x;
  if (b < g.nb && !g.status[b]) g.count[b] += 1;
}

// Complex transpose of nf fields: dst[f][c][r] = src[f][r][c] (rows x cols).
__global__ void k_transpose(const double2* __restrict__ src, double2* __restrict__ dst, int rows,
                            int cols) {
  __shared__ double2 t[32][33];
  const int f = blockIdx.z;
  const size_t off = (size_t)f * rows * cols;
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) t[i][threadIdx.x] = src[off + (size_t)r * cols + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < rows && c < cols) dst[off + (size_t)c * rows + r] = t[threadIdx.x][i];
  }
}

// ------------------------------------------------------------ diagnostics
__device__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
  }
  return s;  // valid in thread 0
}

__device__ double2 warp_sum2(double2 v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// Diagnostics of one step, per member, as tiles (kTiles blocks per member)
// with partial results in part[member][tile][kPart] reduced in a fixed
// order (deterministic):
//   DY: (u, v) on Me >= 2N-1 Gauss points (Fourier modes); DT, DV:
//       c_xx + c_yy on the unpadded Gauss-Lobatto rows (modes, then values).
//   E = <|u|^2/2> by Fejer's first rule in y (exact for degree 2N-2) and
//   Parseval in x; extrema of Tr c = c_xx + c_yy + 1; a non-finite test of
//   the state on the bit patterns; then the counts of Tr c < 3, < 0 and the
//   tie bands |Tr c - 3|, |Tr c| <= tau = 1e-9 max|Tr c|.
enum { P_E = 0, P_MIN, P_MAX, P_AMAX, P_BAD, P_C3, P_C0, P_B3, P_B0 };

__device__ __forceinline__ bool nonfinite(double x) {
  return (__double_as_longlong(x) & 0x7ff0000000000000LL) == 0x7ff0000000000000LL;
}

// block-wide (sum, min, max, max, or) reduction, result valid in thread 0
struct Red5 { double s, mn, mx, ma; int bad; };
__device__ Red5 block_red5(Red5 r) {
  __shared__ double ss[32], smn[32], smx[32], sma[32];
  __shared__ int sbad[32];
  for (int o = 16; o > 0; o >>= 1) {
    r.s += __shfl_down_sync(0xffffffffu, r.s, o);
    r.mn = fmin(r.mn, __shfl_down_sync(0xffffffffu, r.mn, o));
    r.mx = fmax(r.mx, __shfl_down_sync(0xffffffffu, r.mx, o));
    r.ma = fmax(r.ma, __shfl_down_sync(0xffffffffu, r.ma, o));
    r.bad |= __shfl_down_sync(0xffffffffu, r.bad, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) { ss[w] = r.s; smn[w] = r.mn; smx[w] = r.mx; sma[w] = r.ma; sbad[w] = r.bad; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
      r.s += ss[i]; r.mn = fmin(r.mn, smn[i]); r.mx = fmax(r.mx, smx[i]);
      r.ma = fmax(r.ma, sma[i]); r.bad |= sbad[i];
    }
  }
  return r;
}

__global__ void __launch_bounds__(256) k_diag_part(GroupDev g) {
  const int b = blockIdx.y, tile = blockIdx.x;
  if (g.status[b]) return;
  const int K = g.K, N = g.N, nx = g.nx, Je = g.Me;
  const size_t NK = (size_t)N * K;
  const double2* DY = g.DY + (size_t)b * 2 * Je * K;
  Red5 r{0.0, 1e308, -1e308, 0.0, 0};
  // energy: DY fields 0 (u) and 1 (v) on the Me Gauss points (Fejer weights)
  {
    const long long tot = (long long)Je * K, per = (tot + kTiles - 1) / kTiles;
    const long long i0 = tile * per, i1 = min(tot, i0 + per);
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      const int j = (int)(i / K), m = (int)(i - (long long)j * K);
      const double2 uu = DY[i], vv = DY[(size_t)Je * K + i];
      const double w = (m == 0 ? 1.0 : 2.0) * g.ccw[j];
      r.s += w * (uu.x * uu.x + uu.y * uu.y + vv.x * vv.x + vv.y * vv.y);
    }
  }
  // extrema of Tr c on the unpadded grid
  {
    const double* tr = g.DV + (size_t)b * N * nx;
    const long long tot = (long long)N * nx, per = (tot + kTiles - 1) / kTiles;
    const long long i0 = tile * per, i1 = min(tot, i0 + per);
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      const double t = tr[i] + 1.0;
      r.bad |= nonfinite(t);
      r.mn = fmin(r.mn, t);
      r.mx = fmax(r.mx, t);
      r.ma = fmax(r.ma, fabs(t));
    }
  }
  // non-finite state values (integer test)
  {
    const double* X = reinterpret_cast<const double*>(g.X + (size_t)b * 5 * NK);
    const long long tot = 10LL * NK, per = (tot + kTiles - 1) / kTiles;
    const long long i0 = tile * per, i1 = min(tot, i0 + per);
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) r.bad |= nonfinite(X[i]);
  }
  r = block_red5(r);
  if (threadIdx.x == 0) {
    double* pp = g.part + ((size_t)b * kTiles + tile) * kPart;
    pp[P_E] = r.s;
    pp[P_MIN] = r.mn;
    pp[P_MAX] = r.mx;
    pp[P_AMAX] = r.ma;
    pp[P_BAD] = r.bad ? 1.0 : 0.0;
  }
}

__global__ void __launch_bounds__(256) k_diag_count(GroupDev g) {
  const int b = blockIdx.y, tile = blockIdx.x;
  if (g.status[b]) return;
  const int N = g.N, nx = g.nx;
  double ma = 0.0;
  for (int t = 0; t < kTiles; ++t) ma = fmax(ma, g.part[((size_t)b * kTiles + t) * kPart + P_AMAX]);
  const double tau = 1e-9 * ma;
  const double* tr = g.DV + (size_t)b * N * nx;
  const long long tot = (long long)N * nx, per = (tot + kTiles - 1) / kTiles;
  const long long i0 = tile * per, i1 = min(tot, i0 + per);
  int c3 = 0, c0 = 0, b3 = 0, b0 = 0;
  for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const double t = tr[i] + 1.0;
    c3 += (t < 3.0);
    c0 += (t < 0.0);
    b3 += (fabs(t - 3.0) <= tau);
    b0 += (fabs(t) <= tau);
  }
  for (int o = 16; o > 0; o >>= 1) {
    c3 += __shfl_down_sync(0xffffffffu, c3, o);
    c0 += __shfl_down_sync(0xffffffffu, c0, o);
    b3 += __shfl_down_sync(0xffffffffu, b3, o);
    b0 += __shfl_down_sync(0xffffffffu, b0, o);
  }
  __shared__ int sc[4][32];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sc[0][w] = c3; sc[1][w] = c0; sc[2][w] = b3; sc[3][w] = b0; }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t4[4] = {0, 0, 0, 0};
    for (int q = 0; q < 4; ++q)
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t4[q] += sc[q][i];
    double* pp = g.part + ((size_t)b * kTiles + tile) * kPart;
    pp[P_C3] = (double)t4[0];
    pp[P_C0] = (double)t4[1];
    pp[P_B3] = (double)t4[2];
    pp[P_B0] = (double)t4[3];
  }
}

// Mid-plane spectra at y = 0, one warp per (member, Fourier mode):
// T_n(0) = cos(n pi/2), T_n'(0) = n sin(n pi/2).  DM[b][q][m], q = Tr c, u, v,
// du/dy (Chebyshev sums; x derivatives and the mean are applied later).
__global__ void __launch_bounds__(256) k_diag_mid(GroupDev g) {
  const int b = blockIdx.y;
  if (g.status[b]) return;
  const int m = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const int K = g.K, N = g.N;
  if (m >= K) return;
  const size_t NK = (size_t)N * K;
  const double2* X = g.X + (size_t)b * 5 * NK + (size_t)m * N;
  double2 tr = czero(), u = czero(), v = czero(), uy = czero();
  for (int n = lane; n < N; n += 32) {
    const int r4 = n & 3;
    if (r4 == 0 || r4 == 2) {
      const double s = (r4 == 0) ? 1.0 : -1.0;
      tr = cfma(s, cadd(X[2 * NK + n], X[4 * NK + n]), tr);
      u = cfma(s, X[n], u);
      v = cfma(s, X[NK + n], v);
    } else {
      const double s = (r4 == 1) ? (double)n : -(double)n;
      uy = cfma(s, X[n], uy);
    }
  }
  tr = warp_sum2(tr);
  u = warp_sum2(u);
  v = warp_sum2(v);
  uy = warp_sum2(uy);
  if (lane == 0) {
    double2* D = g.DM + (size_t)b * 4 * K + m;
    D[0] = tr;
    D[K] = u;
    D[2 * K] = v;
    D[3 * K] = uy;
  }
}

// Per member: reduce the tiles, <Tr c> from the mean mode, mid-plane
// statistics, blow-up test, record.
__global__ void __launch_bounds__(256) k_diag_final(GroupDev g) {
  const int b = blockIdx.x;
  if (g.status[b]) return;
  __shared__ double sh[32];
  extern __shared__ double2 dsm[];
  const int K = g.K, N = g.N, nx = g.nx;
  const size_t NK = (size_t)N * K;
  const MemberPrm pr = g.prm[b];
  const double* pp = g.part + (size_t)b * kTiles * kPart;
  double tau;
  {
    double ma = 0.0;
    for (int t = 0; t < kTiles; ++t) ma = fmax(ma, pp[t * kPart + P_AMAX]);
    tau = 1e-9 * ma;
  }
  const double2* X = g.X + (size_t)b * 5 * NK;
  // <Tr c> = 1/2 int (c_xx + c_yy)_0 dy + 1, int T_n = 2/(1-n^2), n even
  double mt = 0.0;
  for (int n = threadIdx.x; n < N; n += blockDim.x)
    if ((n & 1) == 0) mt += (X[2 * NK + n].x + X[4 * NK + n].x) * (2.0 / (1.0 - (double)n * n));
  mt = block_sum(mt, sh);
  // mid-plane lines from the per-mode sums: (Tr c, u') (v, du/dx) (dv/dx, du/dy)
  double2* L = dsm;              // 3 lines of nx
  double2* L2 = dsm + 3 * nx;    // ping-pong
  const double kfac = 2.0 * 3.14159265358979323846 / pr.lx;
  for (int i = threadIdx.x; i < 3 * nx; i += blockDim.x) L[i] = czero();
  __syncthreads();
  const double2* DM = g.DM + (size_t)b * 4 * K;
  for (int m = threadIdx.x; m < K; m += blockDim.x) {
    double2 tr = DM[m], u = DM[K + m], v = DM[2 * K + m], uy = DM[3 * K + m];
    const double km = kfac * m;
    double2 ux = cscl(mul_i(u), km), vx = cscl(mul_i(v), km);
    if (m == 0) { tr.x += 1.0; u = czero(); tr.y = v.y = uy.y = 0.0; ux = vx = czero(); }
    const double2 F[6] = {tr, u, v, ux, vx, uy};
    for (int l = 0; l < 3; ++l) {
      L[l * nx + m] = cadd(F[2 * l], mul_i(F[2 * l + 1]));
      if (m > 0) L[l * nx + nx - m] = cadd(cconj(F[2 * l]), mul_i(cconj(F[2 * l + 1])));
    }
  }
  __syncthreads();
  double2* res = fft_lines<+1>(L, L2, 3, nx, g.plNx);
  double sums[6][4];
  long long m3 = 0, m0 = 0, mb3 = 0, mb0 = 0;
  for (int q = 0; q < 6; ++q) for (int k = 0; k < 4; ++k) sums[q][k] = 0.0;
  for (int x = threadIdx.x; x < nx; x += blockDim.x) {
    double q[6];
    for (int l = 0; l < 3; ++l) { q[2 * l] = res[l * nx + x].x; q[2 * l + 1] = res[l * nx + x].y; }
    m3 += (q[0] < 3.0); m0 += (q[0] < 0.0);
    mb3 += (fabs(q[0] - 3.0) <= tau); mb0 += (fabs(q[0]) <= tau);
    for (int qq = 0; qq < 6; ++qq) {
      const double a = q[qq], a2 = a * a;
      sums[qq][0] += a; sums[qq][1] += a2; sums[qq][2] += a2 * a; sums[qq][3] += a2 * a2;
    }
  }
  double msum[6][4];
  for (int qq = 0; qq < 6; ++qq) for (int k = 0; k < 4; ++k) msum[qq][k] = block_sum(sums[qq][k], sh);
  double mc[4] = {(double)m3, (double)m0, (double)mb3, (double)mb0};
  double mct[4];
  for (int q = 0; q < 4; ++q) mct[q] = block_sum(mc[q], sh);
  if (threadIdx.x == 0) {
    double e = 0.0, mn = 1e308, mx = -1e308, c4[4] = {0, 0, 0, 0};
    bool bad = false;
    for (int t = 0; t < kTiles; ++t) {
      const double* q = pp + t * kPart;
      e += q[P_E];
      mn = fmin(mn, q[P_MIN]);
      mx = fmax(mx, q[P_MAX]);
      bad |= (q[P_BAD] != 0.0);
      for (int k = 0; k < 4; ++k) c4[k] += q[P_C3 + k];
    }
    e *= 0.25;
    const long long step = g.count[b];
    const double qnan = __longlong_as_double(0x7ff8000000000000LL);
    ptt_diag r;
    r.step = step;
    r.t = step * pr.dt;
    r.energy = e;
    r.mean_trc = 0.5 * mt + 1.0;
    r.min_trc = bad ? qnan : mn;
    r.max_trc = bad ? qnan : mx;
    r.n_lt3 = (long long)c4[0]; r.n_lt0 = (long long)c4[1];
    r.n_band3 = (long long)c4[2]; r.n_band0 = (long long)c4[3];
    r.n_mid_lt3 = (long long)mct[0]; r.n_mid_lt0 = (long long)mct[1];
    r.n_mid_band3 = (long long)mct[2]; r.n_mid_band0 = (long long)mct[3];
    for (int qq = 0; qq < 8; ++qq)
      for (int k = 0; k < 4; ++k) r.mid_sums[qq][k] = (qq < 6) ? msum[qq][k] : 0.0;
    const bool blow = bad || !isfinite(e) || r.max_trc > pr.trc_max || sqrt(2.0 * e) > pr.u_max;
    r.status = blow ? PTT_BLOWUP : PTT_OK;
    r.reserved = 0;
    g.ring[(size_t)b * kRing + (size_t)(step % kRing)] = r;
    if (blow) g.status[b] = 1;
  }
}

__global__ void k_reset(GroupDev g, int b) {
  if (threadIdx.x == 0) {
    g.count[b] = 0;
    g.status[b] = 0;
  }
}

inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// Spectral coefficients (internal layout [member][field][m][n]) <-> values on
// a y grid stored [member][field][j][m].
YJob make_yjob(const GroupDev& g, bool inverse, int M, int C, const FftPlan& pl,
               const double2* tw4 = nullptr) {
  YJob J{};
  J.gauss = tw4 ? 1 : 0;
  J.tw4 = tw4;
  J.tw4f = g.tw4Pf;
  J.K = g.K;
  J.N = g.N;
  J.M = M;
  J.inverse = inverse ? 1 : 0;
  J.C = C;
  J.pl = pl;
  J.status = g.status;
  J.cm = g.N;
  J.cn = 1;
  J.vm = 1;
  J.vj = g.K;
  for (int i = 0; i < 8; ++i) J.src_field2[i] = -1;
  return J;
}

}  // namespace

size_t smem_ycols(int C, int P, int f32) {
  return (size_t)(2 * C * P + 2 * C) * (f32 ? sizeof(float2) : sizeof(double2));
}
size_t smem_xfused(int Mx, int f32) { return (size_t)14 * Mx * (f32 ? sizeof(float2) : sizeof(double2)); }
size_t smem_xrows(int nl, int n) { return (size_t)2 * nl * n * sizeof(double2); }
size_t smem_spec(int N) { return (size_t)12 * N * sizeof(double2) + (size_t)10 * N * sizeof(double); }

template <typename F>
static cudaError_t optin(F* fn, int optin_bytes) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, fn);
  if (e) return e;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin_bytes - (int)a.sharedSizeBytes);
}

cudaError_t set_kernel_attributes(int optin_bytes) {
  cudaError_t e;
  if ((e = optin(k_ycols<double2>, optin_bytes))) return e;
  if ((e = optin(k_ycols<float2>, optin_bytes))) return e;
  if ((e = optin(k_xfused<double2>, optin_bytes))) return e;
  if ((e = optin(k_xfused<float2>, optin_bytes))) return e;
  if ((e = optin(k_xrows, optin_bytes))) return e;
  if ((e = optin(k_spec, optin_bytes))) return e;
  if ((e = optin(k_diag_final, optin_bytes))) return e;
  return cudaSuccess;
}

// Stage s of one step for one group (see ptt.h: PTT_NSTAGES).
cudaError_t launch_stage(const GroupDev& g, int stage, cudaStream_t st, int* nl) {
  const int rows = g.M;
  const size_t NK = (size_t)g.N * g.K;
  int n = 0;
  switch (stage) {
    case 0: {  // inverse y: 9 fields on the padded Gauss grid (two launches: 8 + 1)
      YJob J = make_yjob(g, true, g.M, g.Ccol, g.plP, g.tw4P);
      J.src = g.X; J.dst = g.f32 ? (void*)g.Ypf : (void*)g.Yp;
      J.dst_f32 = g.f32;
      J.src_mstride = 5 * NK; J.dst_mstride = 9LL * rows * g.K;
      J.src_fstride = NK; J.dst_fstride = (long long)rows * g.K;
      const int sf[9] = {0, 1, 0, 2, 3, 4, 2, 3, 4};
      const int dv[9] = {0, 0, 1, 0, 0, 0, 1, 1, 1};
      for (int i = 0; i < 8; ++i) { J.src_field[i] = sf[i]; J.dst_field[i] = i; J.deriv[i] = dv[i]; }
      YJob J2 = J;
      J2.src_field[0] = sf[8]; J2.dst_field[0] = 8; J2.deriv[0] = dv[8];
      const size_t sm = smem_ycols(g.Ccol, g.M, g.f32);
      if (g.f32) {
        k_ycols<float2><<<dim3(cdiv(g.K, g.Ccol), 8, g.nb), 256, sm, st>>>(J);
        k_ycols<float2><<<dim3(cdiv(g.K, g.Ccol), 1, g.nb), 256, sm, st>>>(J2);
      } else {
        k_ycols<double2><<<dim3(cdiv(g.K, g.Ccol), 8, g.nb), 256, sm, st>>>(J);
        k_ycols<double2><<<dim3(cdiv(g.K, g.Ccol), 1, g.nb), 256, sm, st>>>(J2);
      }
      n = 2;
      break;
    }
    case 1:
      if (g.f32) k_xfused<float2><<<dim3(rows, g.nb), 512, smem_xfused(g.Mx, 1), st>>>(g);
      else k_xfused<double2><<<dim3(rows, g.nb), 512, smem_xfused(g.Mx, 0), st>>>(g);
      n = 1;
      break;
    case 2: {  // forward y of the 5 explicit fields
      YJob F = make_yjob(g, false, g.M, g.Ccol, g.plP, g.tw4P);
      F.src = g.f32 ? (const void*)g.Zpf : (const void*)g.Zp; F.dst = g.NR;
      F.src_f32 = g.f32;
      F.src_mstride = 5LL * rows * g.K; F.dst_mstride = 5 * NK;
      F.src_fstride = (long long)rows * g.K; F.dst_fstride = NK;
      for (int i = 0; i < 5; ++i) { F.src_field[i] = i; F.dst_field[i] = i; F.deriv[i] = 0; }
      const size_t sm = smem_ycols(g.Ccol, g.M, g.f32);
      if (g.f32) k_ycols<float2><<<dim3(cdiv(g.K, g.Ccol), 5, g.nb), 256, sm, st>>>(F);
      else k_ycols<double2><<<dim3(cdiv(g.K, g.Ccol), 5, g.nb), 256, sm, st>>>(F);
      n = 1;
      break;
    }
    case 3:
      k_spec<<<dim3(g.K, g.nb), 256, smem_spec(g.N), st>>>(g, 0);
      k_tick<<<cdiv(g.nb, 128), 128, 0, st>>>(g);
      n = 2;
      break;
    case 4: {  // diagnostics
      // c_xx + c_yy on the unpadded Gauss-Lobatto rows (DCT-I), then x
      YJob T = make_yjob(g, true, g.N - 1, g.CcolU, g.plPu);
      T.src = g.X; T.dst = g.DT;
      T.src_mstride = 5 * NK; T.dst_mstride = (long long)NK;
      T.src_fstride = NK; T.dst_fstride = 0;
      T.src_field[0] = 2; T.src_field2[0] = 4; T.dst_field[0] = 0; T.deriv[0] = 0;
      k_ycols<double2><<<dim3(cdiv(g.K, g.CcolU), 1, g.nb), 256, smem_ycols(g.CcolU, g.Pu, 0), st>>>(T);
      // u, v on the Me Gauss points of the energy quadrature
      YJob J = make_yjob(g, true, g.Me, g.CcolE, g.plPe, g.tw4E);
      J.src = g.X; J.dst = g.DY;
      J.src_mstride = 5 * NK; J.dst_mstride = 2LL * g.Me * g.K;
      J.src_fstride = NK; J.dst_fstride = (long long)g.Me * g.K;
      for (int i = 0; i < 2; ++i) { J.src_field[i] = i; J.dst_field[i] = i; J.deriv[i] = 0; }
      k_ycols<double2><<<dim3(cdiv(g.K, g.CcolE), 2, g.nb), 256, smem_ycols(g.CcolE, g.Me, 0), st>>>(J);
      XJob X{};
      X.srcC = g.DT; X.dstR = g.DV;
      X.src_mstride = (long long)NK; X.dst_mstride = (long long)g.N * g.nx;
      X.src_fstride = 0; X.dst_fstride = 0;
      X.src_rstep = 1; X.dst_rstep = 1;
      X.nf = 1; X.K = g.K; X.n = g.nx; X.c2r = 1; X.status = g.status; X.pl = g.plNx;
      k_xrows<<<dim3(g.N, g.nb), 256, smem_xrows(1, g.nx), st>>>(X);
      k_diag_part<<<dim3(kTiles, g.nb), 256, 0, st>>>(g);
      k_diag_count<<<dim3(kTiles, g.nb), 256, 0, st>>>(g);
      k_diag_mid<<<dim3(cdiv(g.K, 8), g.nb), 256, 0, st>>>(g);
      k_diag_final<<<g.nb, 256, smem_xrows(3, g.nx), st>>>(g);
      n = 7;
      break;
    }
    default:
      return cudaErrorInvalidValue;
  }
  if (nl) *nl += n;
  return cudaGetLastError();
}

cudaError_t launch_explicit(const GroupDev& g, cudaStream_t st) {
  for (int s = 0; s < 3; ++s) {
    cudaError_t e = launch_stage(g, s, st, nullptr);
    if (e) return e;
  }
  k_spec<<<dim3(g.K, g.nb), 256, smem_spec(g.N), st>>>(g, 1);
  return cudaGetLastError();
}

cudaError_t launch_step(const GroupDev& g, cudaStream_t st, int* nl) {
  for (int s = 0; s < 4; ++s) {
    cudaError_t e = launch_stage(g, s, st, nl);
    if (e) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_diag(const GroupDev& g, cudaStream_t st, int* nl) {
  return launch_stage(g, 4, st, nl);
}

cudaError_t launch_reset_member(const GroupDev& g, int b, cudaStream_t st) {
  k_reset<<<1, 32, 0, st>>>(g, b);
  return cudaGetLastError();
}

cudaError_t launch_transpose(const double2* src, double2* dst, int nf, int rows, int cols,
                             cudaStream_t st) {
  k_transpose<<<dim3(cdiv(cols, 32), cdiv(rows, 32), nf), dim3(32, 8), 0, st>>>(src, dst, rows, cols);
  return cudaGetLastError();
}

cudaError_t launch_phys_to_state(const GroupDev& g, int b, cudaStream_t st) {
  const size_t NK = (size_t)g.N * g.K;
  // x analysis of 5 fields, each row l -> stageS[f][l][m]
  XJob X{};
  X.srcR = g.stage; X.dstC = g.stageS;
  X.src_fstride = (long long)g.N * g.nx; X.dst_fstride = NK;
  X.src_rstep = 1; X.dst_rstep = 1;
  X.nf = 5; X.K = g.K; X.n = g.nx; X.c2r = 0; X.status = nullptr; X.pl = g.plNx;
  k_xrows<<<dim3(g.N, 1), 256, smem_xrows(3, g.nx), st>>>(X);
  // y analysis (DCT-I on the N Gauss-Lobatto points) -> X of member b
  YJob J = make_yjob(g, false, g.N - 1, g.CcolU, g.plPu);
  J.status = nullptr;
  J.src = g.stageS; J.dst = g.X + (size_t)b * 5 * NK;
  J.src_fstride = NK; J.dst_fstride = NK;
  for (int i = 0; i < 5; ++i) { J.src_field[i] = i; J.dst_field[i] = i; J.deriv[i] = 0; }
  k_ycols<double2><<<dim3(cdiv(g.K, g.CcolU), 5, 1), 256, smem_ycols(g.CcolU, g.Pu, 0), st>>>(J);
  k_reset<<<1, 32, 0, st>>>(g, b);
  return cudaGetLastError();
}

cudaError_t launch_state_to_phys(const GroupDev& g, int b, cudaStream_t st) {
  const size_t NK = (size_t)g.N * g.K;
  YJob J = make_yjob(g, true, g.N - 1, g.CcolU, g.plPu);
  J.status = nullptr;
  J.src = g.X + (size_t)b * 5 * NK; J.dst = g.stageS;
  J.src_fstride = NK; J.dst_fstride = NK;
  for (int i = 0; i < 5; ++i) { J.src_field[i] = i; J.dst_field[i] = i; J.deriv[i] = 0; }
  k_ycols<double2><<<dim3(cdiv(g.K, g.CcolU), 5, 1), 256, smem_ycols(g.CcolU, g.Pu, 0), st>>>(J);
  XJob X{};
  X.srcC = g.stageS; X.dstR = g.stage;
  X.src_fstride = NK; X.dst_fstride = (long long)g.N * g.nx;
  X.src_rstep = 1; X.dst_rstep = 1;
  X.nf = 5; X.K = g.K; X.n = g.nx; X.c2r = 1; X.status = nullptr; X.pl = g.plNx;
  k_xrows<<<dim3(g.N, 1), 256, smem_xrows(3, g.nx), st>>>(X);
  return cudaGetLastError();
}

}  // namespace ptt
