// Device building blocks shared by the 2D and 3D kernels of the sPTT channel
// step: complex arithmetic in double and single precision, mixed-radix
// Stockham FFTs in shared memory, SBDF coefficients, warp-cooperative
// Chebyshev recurrences and quasi-tridiagonal tau sweeps, the Chebyshev
// column transforms (Gauss and Gauss-Lobatto grids) and the Fourier row
// transforms.  Included by each kernel translation unit (internal linkage).
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "ptt_ds.cuh"
#include "ptt_internal.h"

namespace ptt {
namespace {

// Block coordinates of one launch, explicit so that a kernel body can also
// run as one block of a launch over several shape groups (MultiMap).
struct Blk {
  int x, y, z;
};
__device__ __forceinline__ Blk this_blk() { return Blk{(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z}; }

// One launch over the shape groups of a context: group q contributes
// gx[q] * gy[q] * gz[q] blocks, numbered from start[q] in x-fastest order,
// so that each group's blocks see the coordinates of its own launch.
constexpr int kMaxGroupsMulti = 64;
struct MultiMap {
  int ng;
  int gid[kMaxGroupsMulti];      // index of entry q among the context's groups
  int gx[kMaxGroupsMulti], gy[kMaxGroupsMulti], gz[kMaxGroupsMulti];
  unsigned start[kMaxGroupsMulti + 1];
};
// The group of this block (its index among the context's groups) and the
// block's coordinates within that group's launch.
__device__ __forceinline__ int multi_locate(const MultiMap& mm, Blk& bk) {
  const unsigned v = blockIdx.x;
  int lo = 0, hi = mm.ng - 1;   // the entry q with start[q] <= v < start[q + 1]
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (mm.start[mid] <= v) lo = mid; else hi = mid - 1;
  }
  const unsigned l = v - mm.start[lo];
  const unsigned gx = (unsigned)mm.gx[lo], gy = (unsigned)mm.gy[lo];
  bk.x = (int)(l % gx);
  bk.y = (int)((l / gx) % gy);
  bk.z = (int)(l / (gx * gy));
  return mm.gid[lo];
}

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

// compute types: double2 (FP64 path), float2 (mixed path), dsc (double-single:
// the FP64-accurate path on the FP32 pipe, PTT_FP64_DS; see ptt_ds.cuh)
template <typename C2> struct RealOf;
template <> struct RealOf<double2> { using T = double; };
template <> struct RealOf<float2> { using T = float; };
template <> struct RealOf<dsc> { using T = dsf; };
template <typename C2> __device__ __forceinline__ C2 zero2();
template <> __device__ __forceinline__ double2 zero2<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 zero2<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ dsc zero2<dsc>() { return mk_dsc(dsf(0.f, 0.f), dsf(0.f, 0.f)); }
template <typename D> __device__ __forceinline__ D cvt2(double2 v);
template <typename D> __device__ __forceinline__ D cvt2(float2 v);
template <typename D> __device__ __forceinline__ D cvt2(dsc v);
template <> __device__ __forceinline__ double2 cvt2<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 cvt2<float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }
template <> __device__ __forceinline__ double2 cvt2<double2>(float2 v) { return make_double2(v.x, v.y); }
template <> __device__ __forceinline__ float2 cvt2<float2>(float2 v) { return v; }
template <> __device__ __forceinline__ dsc cvt2<dsc>(double2 v) { return dsc_from_double2(v); }
template <> __device__ __forceinline__ dsc cvt2<dsc>(float2 v) {
  return mk_dsc(dsf(v.x, 0.f), dsf(v.y, 0.f));
}
template <> __device__ __forceinline__ dsc cvt2<dsc>(dsc v) { return v; }
template <> __device__ __forceinline__ double2 cvt2<double2>(dsc v) { return dsc_to_double2(v); }
template <> __device__ __forceinline__ float2 cvt2<float2>(dsc v) {
  return make_float2(__fadd_rn(v.x.h, v.x.l), __fadd_rn(v.y.h, v.y.l));
}

// ------------------------------------------- mean / fluctuation products
// The mixed form's products split every field on the padded grid into its
// mean over the periodic directions, a(y), and the fluctuation a'.  The
// products' mean part (a b with both means) is the same at every point of a
// row and is formed once per row in FP64; at each point only the
// fluctuation part a b' + a' b + a' b' is formed, in FP32 with the means
// rounded to FP32 as multipliers.  The FP32 rounding then scales with the
// fluctuations, not with the O(10^4) stretch components of the base state.
// mfl carries (mean as FP32 multiplier, fluctuation) through the same
// product code as the plain types; only its fluctuation part is used.
struct mfl {
  float m, f;
  mfl() = default;
  __host__ __device__ constexpr mfl(float m_, float f_) : m(m_), f(f_) {}
  __host__ __device__ constexpr mfl(int v) : m((float)v), f(0.f) {}        // a constant
  __host__ __device__ explicit constexpr mfl(double v) : m((float)v), f(0.f) {}
};
__device__ __forceinline__ mfl operator+(mfl a, mfl b) { return mfl(a.m + b.m, a.f + b.f); }
__device__ __forceinline__ mfl operator-(mfl a, mfl b) { return mfl(a.m - b.m, a.f - b.f); }
__device__ __forceinline__ mfl operator-(mfl a) { return mfl(-a.m, -a.f); }
__device__ __forceinline__ mfl operator*(mfl a, mfl b) {
  return mfl(a.m * b.m, fmaf(a.m, b.f, fmaf(a.f, b.m, a.f * b.f)));
}
__device__ __forceinline__ mfl& operator+=(mfl& a, mfl b) { a = a + b; return a; }

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

// Radix 8 (the FP32 plans; the FP64 plans keep radices up to 5 and their
// tangent-form twiddles, the double-single ones too: there the eight
// double-single values per butterfly cost more registers than the saved
// pass gains, measured): with w = exp(DIR 2 pi i / 8),
// a_r = v_r + v_{r+4}, b_r = (v_r - v_{r+4}) w^r (r < 4), the even outputs
// are the 4-point DFT of a and the odd ones that of b:
//   y_{2k} = sum_r a_r w^{2rk},  y_{2k+1} = sum_r b_r w^{2rk}.
template <int DIR> struct Bfly<DIR, 8> {
  template <typename C2>
  static __device__ __forceinline__ void run(C2* v) {
    using T = typename RealOf<C2>::T;
    const T h = (T)0.70710678118654752440;   // cos(pi/4)
    C2 a[4], b[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      a[r] = cadd(v[r], v[r + 4]);
      b[r] = csub(v[r], v[r + 4]);
    }
    // w = (1 + DIR i)/sqrt 2, w^2 = DIR i, w^3 = (-1 + DIR i)/sqrt 2
    {
      const C2 ib1 = mul_i(b[1]), ib3 = mul_i(b[3]);
      if (DIR > 0) {
        b[1] = cscl(cadd(b[1], ib1), h);
        b[2] = mul_i(b[2]);
        b[3] = cscl(csub(ib3, b[3]), h);
      } else {
        b[1] = cscl(csub(b[1], ib1), h);
        C2 t;
        t.x = b[2].y;
        t.y = -b[2].x;
        b[2] = t;
        const C2 s3 = cadd(b[3], ib3);
        t.x = -s3.x;
        t.y = -s3.y;
        b[3] = cscl(t, h);
      }
    }
    Bfly<DIR, 4>::run(a);
    Bfly<DIR, 4>::run(b);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[2 * k] = a[k];
      v[2 * k + 1] = b[k];
    }
  }
};

// Odd prime radices 7, 11, 13 (the unpadded lengths nx, 2 (ny - 1) and nz
// may carry one such factor).  With H = (R - 1)/2, t_k = v_k + v_{R-k},
// d_k = v_k - v_{R-k} (k = 1..H) and w = exp(DIR 2 pi i / R):
//   y_0 = v_0 + sum_k t_k,
//   y_j, y_{R-j} = b_j +- i DIR e_j,  b_j = v_0 + sum_k cos(2 pi jk/R) t_k,
//                                     e_j = sum_k sin(2 pi jk/R) d_k  (j = 1..H),
// the cosines and sines of 2 pi m / R (m = 1..H) as literals, the others by
// symmetry (jk reduced mod R).
// cos and sin of 2 pi m / R, m = 1 .. (R - 1)/2 (folded to constants once
// the butterfly's loops are unrolled).
__device__ __forceinline__ constexpr double odd_cos(int R, int m) {
  constexpr double c7[3] = {0.6234898018587335305250, -0.2225209339563144042890, -0.9009688679024191262361};
  constexpr double c11[5] = {0.8412535328311811688618, 0.4154150130018864255292, -0.1423148382732851404438,
                             -0.6548607339452850640569, -0.9594929736144973898904};
  constexpr double c13[6] = {0.8854560256532098959003, 0.5680647467311558025118, 0.1205366802553230533490,
                             -0.3546048870425356259696, -0.7485107481711010986346, -0.9709418174260520271570};
  return R == 7 ? c7[m - 1] : R == 11 ? c11[m - 1] : c13[m - 1];
}
__device__ __forceinline__ constexpr double odd_sin(int R, int m) {
  constexpr double s7[3] = {0.7818314824680298087084, 0.9749279121818236070181, 0.4338837391175581204757};
  constexpr double s11[5] = {0.5406408174555975821076, 0.9096319953545183714117, 0.9898214418809327323760,
                             0.7557495743542582837740, 0.2817325568414296977114};
  constexpr double s13[6] = {0.4647231720437685456560, 0.8229838658936563945796, 0.9927088740980539928007,
                             0.9350162426854148234397, 0.6631226582407952023767, 0.2393156642875577671487};
  return R == 7 ? s7[m - 1] : R == 11 ? s11[m - 1] : s13[m - 1];
}

template <int DIR, int R> struct BflyOdd {
  template <typename C2>
  static __device__ __forceinline__ void run(C2* v) {
    using T = typename RealOf<C2>::T;
    constexpr int H = (R - 1) / 2;
    C2 t[H], d[H];
#pragma unroll
    for (int k = 1; k <= H; ++k) {
      t[k - 1] = cadd(v[k], v[R - k]);
      d[k - 1] = csub(v[k], v[R - k]);
    }
    C2 y[R];
    y[0] = v[0];
#pragma unroll
    for (int k = 0; k < H; ++k) y[0] = cadd(y[0], t[k]);
#pragma unroll
    for (int j = 1; j <= H; ++j) {
      C2 b = v[0], e = zero2<C2>();
#pragma unroll
      for (int k = 1; k <= H; ++k) {
        const int mm = (j * k) % R;                  // 1 .. R-1
        const int mi = (mm <= H) ? mm : R - mm;      // cos even, sin odd about R/2
        const T c = (T)odd_cos(R, mi);
        const T sn = (T)((mm <= H) ? odd_sin(R, mi) : -odd_sin(R, mi));
        b = cfma(c, t[k - 1], b);
        e = cfma(sn, d[k - 1], e);
      }
      const C2 ie = cscl(mul_i(e), (T)DIR);
      y[j] = cadd(b, ie);
      y[R - j] = csub(b, ie);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = y[r];
  }
};
template <int DIR> struct Bfly<DIR, 7> : BflyOdd<DIR, 7> {};
template <int DIR> struct Bfly<DIR, 11> : BflyOdd<DIR, 11> {};
template <int DIR> struct Bfly<DIR, 13> : BflyOdd<DIR, 13> {};

// Division by a runtime divisor d through a multiply-high (the method of
// Granlund and Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994, in its round-up form): with
// m = floor((2^32 - 1)/d) + 1 = ceil(2^32/d), floor(x/d) = (x m) >> 32 holds
// exactly whenever x d < 2^32 (the rounding excess of m contributes less than
// x/2^32 < 1/d), which covers every index of the transforms here
// (x < 2^20, d < 2^12).  d = 1 is passed through.
struct FastDiv {
  unsigned m;
  bool one;
};
__device__ __forceinline__ FastDiv fast_div(unsigned d) {
  FastDiv f;
  f.one = (d == 1u);
  f.m = f.one ? 0u : 0xFFFFFFFFu / d + 1u;
  return f;
}
__device__ __forceinline__ unsigned fdiv(unsigned x, FastDiv f) { return f.one ? x : __umulhi(x, f.m); }

// Constants of pass s of a plan, read from the plan (host-computed): the
// passes divide nothing at run time.
struct PassC {
  int nb, st, Ns;
  FastDiv dnb, dns;
};
__device__ __forceinline__ PassC pass_c(const FftPlan& pl, int s) {
  PassC c;
  c.nb = pl.pnb[s];
  c.st = pl.pst[s];
  c.Ns = pl.pns[s];
  c.dnb = FastDiv{pl.pmb[s], pl.pmb[s] == 0u};
  c.dns = FastDiv{pl.pms[s], pl.pms[s] == 0u};
  return c;
}

// read-only table loads (the double-single table as one 16-byte load)
__device__ __forceinline__ double2 ldg_tw(const double2* p) { return __ldg(p); }
__device__ __forceinline__ float2 ldg_tw(const float2* p) { return __ldg(p); }
__device__ __forceinline__ dsc ldg_tw(const dsc* p) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return mk_dsc(dsf(v.x, v.y), dsf(v.z, v.w));
}

// One Stockham pass of radix R over nl lines (line l at offset l*ls).
template <int DIR, int R, typename C2>
__device__ __forceinline__ void fft_pass(const C2* __restrict__ src, C2* __restrict__ dst,
                                         int nl, int ls, const PassC& c,
                                         const C2* __restrict__ tw) {
  const int nb = c.nb, st = c.st, Ns = c.Ns;
  const int total = nl * nb;
  const FastDiv dnb = c.dnb, dns = c.dns;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int l = (int)fdiv((unsigned)t, dnb);
    const int j = t - l * nb;
    const C2* s = src + l * ls;
    C2* d = dst + l * ls;
    const int jq = (int)fdiv((unsigned)j, dns);
    const int jm = j - jq * Ns;
    C2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = s[j + r * nb];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C2 w = ldg_tw(&tw[jm * r * st]);
        if (DIR > 0) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    Bfly<DIR, R>::run(v);
    const int o = jq * Ns * R + jm;
#pragma unroll
    for (int r = 0; r < R; ++r) d[o + r * Ns] = v[r];
  }
}

// ---------------------------------------------- tangent-form FP64 passes
// A twiddle i^k c (1 + i t) applied as u = v + i t v (two FMAs), the quarter
// turn i^k by swaps and sign flips (integer operations), and c folded into
// the butterfly's sums as FMA coefficients: 6, 16, 22 and 44 FP64 operations
// for a twiddled radix-2, 3, 4 and 5 butterfly against 8, 20, 28 and 52 with
// plain complex products.  Tables: FftPlan::tt, tk.
__device__ __forceinline__ double flip_sign(double v, bool c) {
  return __hiloint2double(__double2hiint(v) ^ (c ? (int)0x80000000 : 0), __double2loint(v));
}
__device__ __forceinline__ double2 rot_quarter(double2 u, int k) {   // i^k u, k in 0..3
  const bool sw = k & 1;
  const double x = sw ? u.y : u.x, y = sw ? u.x : u.y;
  return make_double2(flip_sign(x, k == 1 || k == 2), flip_sign(y, k >= 2));
}
// i^k (1 + i t) v for the forward twiddle; the inverse uses the conjugate,
// i^-k (1 - i t) v.
template <int DIR>
__device__ __forceinline__ double2 tan_rotate(double2 v, double t, int k) {
  if (DIR > 0) { t = -t; k = (4 - k) & 3; }
  return rot_quarter(make_double2(fma(-t, v.y, v.x), fma(t, v.x, v.y)), k);
}

template <int DIR, int R>
__device__ __forceinline__ void fft_pass_tan(const double2* __restrict__ src, double2* __restrict__ dst,
                                             int nl, int ls, const PassC& c,
                                             const double* __restrict__ tt,
                                             const int* __restrict__ tk) {
  const int nb = c.nb, Ns = c.Ns;
  const int total = nl * nb;
  const FastDiv dnb = c.dnb, dns = c.dns;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int l = (int)fdiv((unsigned)t, dnb);
    const int j = t - l * nb;
    const double2* s = src + l * ls;
    double2* d = dst + l * ls;
    const int jq = (int)fdiv((unsigned)j, dns);
    const int jm = j - jq * Ns;
    const double* rec = tt + (size_t)(R == 5 ? 16 : 6) * jm;
    const int kp = tk[jm];
    const int o = jq * Ns * R + jm;
    const double2 v0 = s[j];
    if (R == 2) {
      const double2 u1 = tan_rotate<DIR>(s[j + nb], rec[0], kp & 3);
      const double c1 = rec[1];
      d[o] = make_double2(fma(c1, u1.x, v0.x), fma(c1, u1.y, v0.y));
      d[o + Ns] = make_double2(fma(-c1, u1.x, v0.x), fma(-c1, u1.y, v0.y));
    } else if (R == 3) {
      const double2 u1 = tan_rotate<DIR>(s[j + nb], rec[0], kp & 3);
      const double2 u2 = tan_rotate<DIR>(s[j + 2 * nb], rec[1], (kp >> 2) & 3);
      const double c1 = rec[2], rho = rec[3], h = rec[4], sc = (DIR > 0) ? rec[5] : -rec[5];
      const double2 q = make_double2(fma(rho, u2.x, u1.x), fma(rho, u2.y, u1.y));     // (a1 + a2)/c1
      const double2 qm = make_double2(fma(-rho, u2.x, u1.x), fma(-rho, u2.y, u1.y));  // (a1 - a2)/c1
      const double2 m = make_double2(fma(-h, q.x, v0.x), fma(-h, q.y, v0.y));
      d[o] = make_double2(fma(c1, q.x, v0.x), fma(c1, q.y, v0.y));
      // y1 = m + i s (a1 - a2), y2 = m - i s (a1 - a2), s = DIR sin(2 pi/3)
      d[o + Ns] = make_double2(fma(-sc, qm.y, m.x), fma(sc, qm.x, m.y));
      d[o + 2 * Ns] = make_double2(fma(sc, qm.y, m.x), fma(-sc, qm.x, m.y));
    } else if (R == 5) {
      // a_r = c_r u_r; with t1 = a1 + a4 = c1 q1, d1 = a1 - a4 = c1 m1,
      // t2 = a2 + a3 = c2 q2, d2 = a2 - a3 = c2 m2 the radix-5 DFT reads
      // y0 = v0 + t1 + t2, b1 = v0 + C1 t1 + C2 t2, b2 = v0 + C2 t1 + C1 t2,
      // y1,4 = b1 +- i DIR (S1 d1 + S2 d2), y2,3 = b2 +- i DIR (S2 d1 - S1 d2)
      const double2 u1 = tan_rotate<DIR>(s[j + nb], rec[0], kp & 3);
      const double2 u2 = tan_rotate<DIR>(s[j + 2 * nb], rec[1], (kp >> 2) & 3);
      const double2 u3 = tan_rotate<DIR>(s[j + 3 * nb], rec[2], (kp >> 4) & 3);
      const double2 u4 = tan_rotate<DIR>(s[j + 4 * nb], rec[3], (kp >> 6) & 3);
      const double r14 = rec[4], r23 = rec[5];
      const double2 q1 = make_double2(fma(r14, u4.x, u1.x), fma(r14, u4.y, u1.y));
      const double2 m1 = make_double2(fma(-r14, u4.x, u1.x), fma(-r14, u4.y, u1.y));
      const double2 q2 = make_double2(fma(r23, u3.x, u2.x), fma(r23, u3.y, u2.y));
      const double2 m2 = make_double2(fma(-r23, u3.x, u2.x), fma(-r23, u3.y, u2.y));
      const double c1 = rec[6], c2 = rec[7];
      d[o] = make_double2(fma(c1, q1.x, fma(c2, q2.x, v0.x)), fma(c1, q1.y, fma(c2, q2.y, v0.y)));
      const double2 b1 = make_double2(fma(rec[8], q1.x, fma(rec[9], q2.x, v0.x)),
                                      fma(rec[8], q1.y, fma(rec[9], q2.y, v0.y)));
      const double2 b2 = make_double2(fma(rec[10], q1.x, fma(rec[11], q2.x, v0.x)),
                                      fma(rec[10], q1.y, fma(rec[11], q2.y, v0.y)));
      const double2 e1 = make_double2(fma(rec[12], m1.x, rec[13] * m2.x), fma(rec[12], m1.y, rec[13] * m2.y));
      const double2 e2 = make_double2(fma(rec[14], m1.x, -rec[15] * m2.x), fma(rec[14], m1.y, -rec[15] * m2.y));
      // i e = (-e.y, e.x); DIR < 0: y1 = b1 - i e1, y4 = b1 + i e1 (likewise y2, y3)
      const double2 p1 = make_double2(b1.x - e1.y, b1.y + e1.x), n1 = make_double2(b1.x + e1.y, b1.y - e1.x);
      const double2 p2 = make_double2(b2.x - e2.y, b2.y + e2.x), n2 = make_double2(b2.x + e2.y, b2.y - e2.x);
      d[o + Ns] = (DIR < 0) ? n1 : p1;
      d[o + 4 * Ns] = (DIR < 0) ? p1 : n1;
      d[o + 2 * Ns] = (DIR < 0) ? n2 : p2;
      d[o + 3 * Ns] = (DIR < 0) ? p2 : n2;
    } else {
      const double2 u1 = tan_rotate<DIR>(s[j + nb], rec[0], kp & 3);
      const double2 u2 = tan_rotate<DIR>(s[j + 2 * nb], rec[1], (kp >> 2) & 3);
      const double2 u3 = tan_rotate<DIR>(s[j + 3 * nb], rec[2], (kp >> 4) & 3);
      const double c1 = rec[3], c2 = rec[4], rho = rec[5];
      const double2 s02 = make_double2(fma(c2, u2.x, v0.x), fma(c2, u2.y, v0.y));
      const double2 d02 = make_double2(fma(-c2, u2.x, v0.x), fma(-c2, u2.y, v0.y));
      const double2 q = make_double2(fma(rho, u3.x, u1.x), fma(rho, u3.y, u1.y));     // (a1 + a3)/c1
      const double2 qm = make_double2(fma(-rho, u3.x, u1.x), fma(-rho, u3.y, u1.y));  // (a1 - a3)/c1
      d[o] = make_double2(fma(c1, q.x, s02.x), fma(c1, q.y, s02.y));
      d[o + 2 * Ns] = make_double2(fma(-c1, q.x, s02.x), fma(-c1, q.y, s02.y));
      // d13 = i (a1 - a3) = c1 (-qm.y, qm.x); forward y1 = d02 - d13, y3 = d02 + d13
      const double2 yA = make_double2(fma(c1, qm.y, d02.x), fma(-c1, qm.x, d02.y));   // d02 - d13
      const double2 yB = make_double2(fma(-c1, qm.y, d02.x), fma(c1, qm.x, d02.y));   // d02 + d13
      d[o + Ns] = (DIR < 0) ? yA : yB;
      d[o + 3 * Ns] = (DIR < 0) ? yB : yA;
    }
  }
}

// First pass of radix 3 (no twiddles) for lines that are zero in their
// middle third [n/3, 2n/3) -- the inverse transforms of spectra padded to
// n >= 3K points for K kept modes: with v1 = 0 the butterfly is
// y0 = v0 + v2, y1,2 = v0 - v2/2 -+ DIR sin(2 pi/3) i v2 (8 operations).
template <int DIR, typename C2>
__device__ __forceinline__ void fft_pass_r3_zmid(const C2* __restrict__ src, C2* __restrict__ dst,
                                                 int nl, int ls, const PassC& c) {
  using T = typename RealOf<C2>::T;
  const int nb = c.nb;
  const int total = nl * nb;
  const FastDiv dnb = c.dnb;
  const T sn = (T)(DIR * 0.86602540378443864676);  // sin(2 pi / 3), signed
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int l = (int)fdiv((unsigned)t, dnb);
    const int j = t - l * nb;
    const C2 v0 = src[l * ls + j], v2 = src[l * ls + j + 2 * nb];
    C2 m, y1, y2;
    m.x = fma((T)-0.5, v2.x, v0.x);
    m.y = fma((T)-0.5, v2.y, v0.y);
    y1.x = fma(sn, v2.y, m.x);
    y1.y = fma(-sn, v2.x, m.y);
    y2.x = fma(-sn, v2.y, m.x);
    y2.y = fma(sn, v2.x, m.y);
    C2* d = dst + l * ls + 3 * j;
    d[0] = cadd(v0, v2);
    d[1] = y1;
    d[2] = y2;
  }
}

template <typename C2> __device__ __forceinline__ const C2* plan_tw(const FftPlan& pl);
template <> __device__ __forceinline__ const double2* plan_tw<double2>(const FftPlan& pl) { return pl.tw; }
template <> __device__ __forceinline__ const float2* plan_tw<float2>(const FftPlan& pl) { return pl.twf; }
template <> __device__ __forceinline__ const dsc* plan_tw<dsc>(const FftPlan& pl) {
  return reinterpret_cast<const dsc*>(pl.twd);
}

// Unnormalised DFT of nl lines of length pl.n held in `a`, using `b` as the
// ping-pong buffer.  Returns the buffer holding the result.  Must be called
// by the whole block after a __syncthreads(); ends with one.  zero_mid: the
// lines are zero in their middle third and the plan starts with radix 3.
// BIG: the plan may hold radices 7, 11, 13 (unpadded lengths); without it
// only 2 to 5 are compiled in (the padded lengths, chosen 5-smooth), which
// keeps the register budget of the hot transform kernels, and a pass of
// another radix is skipped (the launch code never gives such a plan).
template <int DIR, typename C2, bool BIG = false>
__device__ C2* fft_lines(C2* a, C2* b, int nl, int ls, const FftPlan& pl, bool zero_mid = false) {
  C2* src = a;
  C2* dst = b;
  const C2* tw = plan_tw<C2>(pl);
  for (int s = 0; s < pl.nst; ++s) {
    const int R = pl.radix[s];
    const PassC c = pass_c(pl, s);
    if (s == 0 && zero_mid && R == 3) {
      fft_pass_r3_zmid<DIR>(src, dst, nl, ls, c);
      __syncthreads();
      C2* t = src; src = dst; dst = t;
      continue;
    }
    if constexpr (std::is_same<C2, double2>::value) {
      if (pl.tt && s > 0 && R <= 5) {
        const double* tt = pl.tt + pl.tto[s];
        const int* tk = pl.tk + pl.toff[s];
        if (R == 5) fft_pass_tan<DIR, 5>(src, dst, nl, ls, c, tt, tk);
        else if (R == 4) fft_pass_tan<DIR, 4>(src, dst, nl, ls, c, tt, tk);
        else if (R == 3) fft_pass_tan<DIR, 3>(src, dst, nl, ls, c, tt, tk);
        else fft_pass_tan<DIR, 2>(src, dst, nl, ls, c, tt, tk);
        __syncthreads();
        C2* t = src; src = dst; dst = t;
        continue;
      }
    }
    switch (R) {
      case 2: fft_pass<DIR, 2>(src, dst, nl, ls, c, tw); break;
      case 3: fft_pass<DIR, 3>(src, dst, nl, ls, c, tw); break;
      case 4: fft_pass<DIR, 4>(src, dst, nl, ls, c, tw); break;
      case 5: fft_pass<DIR, 5>(src, dst, nl, ls, c, tw); break;
      case 8:   // plans of FP32 groups only (see wide_plans); compiled for
                // FP32 alone, so the FP64 and double-single kernels keep
                // their register budgets
        if constexpr (std::is_same<C2, float2>::value) fft_pass<DIR, 8>(src, dst, nl, ls, c, tw);
        break;
      default:
        if constexpr (BIG) {
          if (R == 7) fft_pass<DIR, 7>(src, dst, nl, ls, c, tw);
          else if (R == 11) fft_pass<DIR, 11>(src, dst, nl, ls, c, tw);
          else if (R == 13) fft_pass<DIR, 13>(src, dst, nl, ls, c, tw);
        }
        break;
    }
    __syncthreads();
    C2* t = src; src = dst; dst = t;
  }
  return src;
}

// ---------------------------------------------- in-place FFT passes
// For lines too long for two buffers in shared memory (the FP64 3D x pass
// at Mx = 768): each pass gathers its butterflies' inputs into registers,
// waits for the whole block, and writes the outputs over the same buffer.
// Lines go in groups of at most kIpLines, so that a thread holds at most
// ip_maxb(R) butterflies with blockDim.x = kIpThreads and n <= kIpMaxN.
// Plain twiddles (FftPlan::tw).
constexpr int kIpThreads = 512, kIpLines = 3, kIpMaxN = 768;
__host__ __device__ constexpr int ip_maxb(int R) {
  return (kIpLines * kIpMaxN / R + kIpThreads - 1) / kIpThreads;
}

template <int DIR, int R, typename C2>
__device__ __forceinline__ void fft_pass_ip(C2* a, int nl, int ls, const PassC& c,
                                            const C2* __restrict__ tw, bool zmid) {
  constexpr int MB = ip_maxb(R);
  const int nb = c.nb, st = c.st, Ns = c.Ns;
  const int total = nl * nb;
  const FastDiv dnb = c.dnb, dns = c.dns;
  const int tid = threadIdx.x, nt = blockDim.x;
  C2 v[MB][R];
#pragma unroll
  for (int q = 0; q < MB; ++q) {
    const int t = tid + q * nt;
    if (t < total) {
      const int l = (int)fdiv((unsigned)t, dnb), j = t - l * nb;
      const C2* s = a + l * ls;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = (zmid && r == 1) ? zero2<C2>() : s[j + r * nb];
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < MB; ++q) {
    const int t = tid + q * nt;
    if (t < total) {
      const int l = (int)fdiv((unsigned)t, dnb), j = t - l * nb;
      C2* d = a + l * ls;
      const int jq = (int)fdiv((unsigned)j, dns), jm = j - jq * Ns;
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          C2 w = ldg_tw(&tw[jm * r * st]);
          if (DIR > 0) w.y = -w.y;
          v[q][r] = cmul(v[q][r], w);
        }
      }
      Bfly<DIR, R>::run(v[q]);
      const int o = jq * Ns * R + jm;
#pragma unroll
      for (int r = 0; r < R; ++r) d[o + r * Ns] = v[q][r];
    }
  }
  __syncthreads();
}

// In-place unnormalised DFT of nl lines of length pl.n (radices 2 to 5) in
// `a`; zero_mid as for fft_lines.  Called by the whole block (kIpThreads
// threads) after a __syncthreads(); ends with one.
template <int DIR, typename C2>
__device__ void fft_lines_inplace(C2* a, int nl, int ls, const FftPlan& pl, bool zero_mid = false) {
  const C2* tw = plan_tw<C2>(pl);
  for (int l0 = 0; l0 < nl; l0 += kIpLines) {
    const int g = min(kIpLines, nl - l0);
    C2* base = a + (size_t)l0 * ls;
    for (int s = 0; s < pl.nst; ++s) {
      const int R = pl.radix[s];
      const PassC c = pass_c(pl, s);
      const bool zm = (s == 0 && zero_mid && R == 3);
      switch (R) {
        case 2: fft_pass_ip<DIR, 2>(base, g, ls, c, tw, false); break;
        case 3: fft_pass_ip<DIR, 3>(base, g, ls, c, tw, zm); break;
        case 4: fft_pass_ip<DIR, 4>(base, g, ls, c, tw, false); break;
        default: fft_pass_ip<DIR, 5>(base, g, ls, c, tw, false); break;
      }
    }
  }
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
__constant__ float c_sbf[4][4] = {{1.f, 0.f, 0.f, 0.f},   // the same (exact in FP32)
                                  {2.f, -1.f, 0.f, 0.f},
                                  {3.f, -3.f, 1.f, 0.f},
                                  {4.f, -6.f, 4.f, -1.f}};

// 2D mixed groups keep the explicit-term history and its SBDF sum in FP32
// for every mode but the mean (the explicit terms carry FP32 accuracy there):
// each member's FP32 history sits in the first half of its own block of the
// FP64 history array, the mean mode's FP64 history in the second half (so
// checkpoints copy the same byte ranges).  FP64 <-> FP32 by integer
// operations.
__device__ __forceinline__ float2 f2_trunc(double2 v) {
  return make_float2(ds_from_double(v.x).h, ds_from_double(v.y).h);
}
__device__ __forceinline__ double2 d2_exact(float2 v) {
  return make_double2(ds_f32_to_f64(v.x), ds_f32_to_f64(v.y));
}

// ------------------------------------------- warp-cooperative recurrences
// FP64 runs at a few lanes per clock per SM on this part, so a warp FP64
// instruction costs the same pipe time whether 1 or 32 lanes are active.
// The Chebyshev recurrences and the tau sweeps are therefore written as
// warp scans: each lane takes a contiguous chunk, composes it sequentially,
// and the chunks are combined with shuffles.
constexpr unsigned kFull = 0xffffffffu;
// tau solves: above this top elimination factor the top coefficient of a
// parity is taken from its wall row (see warp_qt_solve)
constexpr double kTopFromWall = 1e3;
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
__device__ void warp_cheb_deriv_par(const C2* a, C2* out, int N, int par) {
  using T = typename RealOf<C2>::T;
  const int lane = threadIdx.x & 31;
  const int L = (N - par + 1) / 2;
  const int c = (L + 31) / 32;
  const int i0 = min(lane * c, L), i1 = min(i0 + c, L);
  // partial sums carried doubled (2 k a_k): b_{k-1} = acc + ex for k >= 2
  // and (acc + ex)/2 for k = 1, with no scaling in the sweeps
  C2 acc = zero2<C2>();
  for (int i = i1 - 1; i >= i0; --i) {
    const int k = par + 2 * i;
    acc = cfma((T)(2 * k), a[k], acc);
    if (k >= 1) out[k - 1] = acc;
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
    if (k >= 2) out[k - 1] = cadd(ex, out[k - 1]);
    else if (k == 1) out[0] = cscl(cadd(ex, out[0]), (T)0.5);
  }
  // out_{N-1} (parity of N - 1) has no term
  if (lane == 0 && ((N - 1 - par) & 1)) out[N - 1] = zero2<C2>();
  __syncwarp();
}

template <typename C2>
__device__ void warp_cheb_deriv(const C2* a, C2* out, int N) {
  warp_cheb_deriv_par(a, out, N, 0);
  warp_cheb_deriv_par(a, out, N, 1);
}

// -x for complex values by sign-bit flips (integer operations, no FP64 work)
__device__ __forceinline__ double2 cneg_bits(double2 v) {
  return make_double2(flip_sign(v.x, true), flip_sign(v.y, true));
}

// Warp-cooperative quasi-tridiagonal tau solve (system stated at k_spec): the backward
// elimination P_i = alpha_i + beta_i P_{i+1} and the forward substitution
// a_i = P_i + Q_i a_{i-1} are affine recurrences, evaluated as warp scans of
// affine maps; the boundary sums are warp reductions.  `out` may alias R.
// CH >= the rows per lane, ceil((L - 1)/32) (register arrays of that size).
template <int CH>
__device__ void warp_qt_solve(int N, int p, double alpha, const double2* R, double2* out,
                              const double* Q, const double* inv, const double* F, double G,
                              const double* w1, const double* w2, const double* w3,
                              double bcfac, double rsign) {
  const int lane = threadIdx.x & 31;
  const int L = (N - p + 1) / 2;  // unknowns a_{p+2i}, i < L; rows i = 1..L-1
  const int nr = L - 1;
  const int c = (nr + 31) / 32;
  const int i0 = min(1 + lane * c, L), i1 = min(i0 + c, L);
  double2 al[CH];
  double be[CH];
  double2 rs = czero();
#pragma unroll
  for (int t = 0; t < CH; ++t) {
    const int i = i0 + t;
    if (t < c && i < i1) {
      const int n = p + 2 * i;
      const double2 Rm2 = R[n - 2];
      const double2 R0 = R[n];
      const double cc = (n == 2) ? 2.0 : 1.0;
      double2 r = cscl(Rm2, -cc * w1[n]);
      if (n <= N - 3) r = cfma(w2[n], R0, r);
      double un = 0.0;
      if (n <= N - 5) {
        r = cfma(-w3[n], R[n + 2], r);
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
  if (lane == 0) rs = cadd(rs, R[p]);
  __syncwarp();
  // backward: chunk map P_{i0} = A + B P_{i1}
  double2 A = czero();
  double B = 1.0;
#pragma unroll
  for (int t = CH - 1; t >= 0; --t) {
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
  for (int t = CH - 1; t >= 0; --t) {
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
  double2 Pv[CH];
  double Qv[CH];
#pragma unroll
  for (int t = 0; t < CH; ++t) {
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
  double2 part = (lane == 0) ? a0 : czero();  // sum of a_{p+2i}, i < L-1
  __syncwarp();
#pragma unroll
  for (int t = 0; t < CH; ++t) {
    const int i = i0 + t;
    if (t < c && i < i1) {
      av = cfma(Qv[t], av, Pv[t]);
      out[p + 2 * i] = av;
      if (i < L - 1) part = cadd(part, av);
    }
  }
  if (lane == 0) out[p] = a0;
  __syncwarp();
  // Top coefficient from the wall row when the top elimination factor is
  // large: with a small diagonal (diffusivity kappa) the forward
  // substitution forms a_top = P + Q a_{top-2} with |Q| ~ alpha/(4 n^2 kappa)
  // and amplifies the rounding of a_{top-2}; the wall row of the same system
  // gives a_top = g - sum of the others with rounding of the sum only.
  const int nl = p + 2 * (L - 1);
  if (L > 1 && fabs(Q[nl]) > kTopFromWall) {
    part = warp_allsum2(part);
    if (lane == 0) out[nl] = csub(cscl(rs, bcfac), part);
    __syncwarp();
  }
  // the solve above is of (alpha - beta D^2) a = R; the system's right-hand
  // side is rsign R, so a flips sign with it
  if (rsign < 0.0) {
    for (int i = lane; i < L; i += 32) out[p + 2 * i] = cneg_bits(out[p + 2 * i]);
    __syncwarp();
  }
}

// Lane-sequential forms for the per-mode spectral stage: one lane owns one
// (Fourier mode, Chebyshev parity) pair and walks its ~N/2 coefficients in
// order, so a warp advances 32 independent recurrences with every lane busy.
// Columns are indexed by n (stride 1); a lane touches only n = p mod 2 on
// input and, for the derivative, only n = 1 - p mod 2 on output.

// Chebyshev derivative, parity half: from the inputs a_k, k = p mod 2, the
// outputs b_{k-1} = (k == 1 ? 1 : 2) sum_{k' >= k, k' = k mod 2} k' a_{k'}
// (b_{n-1} = b_{n+1} + 2 n a_n, b_0 halved); the lane whose output parity is
// that of N - 1 also writes b_{N-1} = 0.  The two lanes of one column
// together produce the whole derivative; `out` must not alias `a`.
__device__ __forceinline__ void lane_cheb_deriv(const double2* __restrict__ a,
                                                double2* __restrict__ out, int N, int p) {
  const int top = ((N - 1 - p) & ~1) + p;   // largest k = p mod 2 below N
  double2 acc = czero();
#pragma unroll 4
  for (int k = top; k >= 1; k -= 2) {
    acc = cfma((double)k, a[k], acc);
    out[k - 1] = cscl(acc, k == 1 ? 1.0 : 2.0);
  }
  if (((N - 1) & 1) != p) out[N - 1] = czero();
}

// Quasi-tridiagonal tau solve of one parity (system stated at k_spec):
// backward elimination P_n = (r_n - u_n P_{n+2}) inv_n with the three-term
// right-hand side r_n of the twice-integrated rows, accumulating the
// boundary sum U = sum F_n P_n; the boundary row gives
// a_p = (bcfac sum_{n = p} R_n - U) G; forward substitution
// a_n = P_n + Q_n a_{n-2}.  Q, inv, F: the right-hand-side-independent
// elimination factors of this (alpha, mode, parity), precomputed on the
// host.  The solve runs on R and flips the result's sign when the system's
// right-hand side is rsign R with rsign = -1.  `out` must not alias R (every
// input is independent of the recurrence, so unrolled iterations keep
// several loads in flight).
__device__ __forceinline__ void lane_qt_solve(int N, int p, double alpha,
                                              const double2* __restrict__ R,
                                              double2* __restrict__ out,
                                              const double* __restrict__ Q,
                                              const double* __restrict__ inv,
                                              const double* __restrict__ F, double G,
                                              const double* __restrict__ w1,
                                              const double* __restrict__ w2,
                                              const double* __restrict__ w3, double bcfac,
                                              double rsign) {
  const int nl = ((N - 1 - p) & ~1) + p;
  double2 Pn2 = czero(), U = czero(), rs = czero(), Rp2 = czero();
  double2 R0 = R[nl];
#pragma unroll 4
  for (int n = nl; n >= p + 2; n -= 2) {
    const double2 Rm2 = R[n - 2];
    const double cc = (n == 2) ? 2.0 : 1.0;
    double2 r = cscl(Rm2, -cc * w1[n]);
    if (n <= N - 3) r = cfma(w2[n], R0, r);
    double un = 0.0;
    if (n <= N - 5) {
      r = cfma(-w3[n], Rp2, r);
      un = -alpha * w3[n];
    }
    const double2 P = cscl(cfma(-un, Pn2, r), inv[n]);
    out[n] = P;
    U = cfma(F[n], P, U);
    rs = cadd(rs, R0);
    Pn2 = P;
    Rp2 = R0;
    R0 = Rm2;
  }
  rs = cadd(rs, R0);   // R_p
  double2 a = cscl(csub(cscl(rs, bcfac), U), G);
  out[p] = a;
#pragma unroll 4
  for (int n = p + 2; n <= nl; n += 2) {
    a = cfma(Q[n], a, out[n]);
    out[n] = a;
  }
  if (nl > p && fabs(Q[nl]) > kTopFromWall) {   // top coefficient from the wall row
    double2 part = czero();
    for (int n = p; n < nl; n += 2) part = cadd(part, out[n]);
    out[nl] = csub(cscl(rs, bcfac), part);
  }
  // solved for R; the right-hand side is rsign R
  if (rsign < 0.0)
    for (int n = p; n <= nl; n += 2) out[n] = cneg_bits(out[n]);
}

// SBDF sum of one evolved column, parity p, order index O (0..3: SBDF1-4):
// writes the current values x, nn into the history slot (E, Nn) and
// R = sb_0 nn + sum_j (-sa_{j+1}/dt) x^{n-j} + sum_{j>=1} sb_j N^{n-j}
// over the O older slots Eo[j-1], No[j-1].
template <int O>
__device__ __forceinline__ void lane_sbdf(int N, int p, double idt,
                                          const double2* __restrict__ x,
                                          const double2* __restrict__ nn,
                                          double2* __restrict__ E, double2* __restrict__ Nn,
                                          const double2* __restrict__ Eo0,
                                          const double2* __restrict__ Eo1,
                                          const double2* __restrict__ Eo2,
                                          const double2* __restrict__ No0,
                                          const double2* __restrict__ No1,
                                          const double2* __restrict__ No2,
                                          double2* __restrict__ R) {
  const double ca0 = -c_sa[O][1] * idt, cb0 = c_sb[O][0];
  const double ca1 = (O >= 1) ? -c_sa[O][2] * idt : 0.0, cb1 = (O >= 1) ? c_sb[O][1] : 0.0;
  const double ca2 = (O >= 2) ? -c_sa[O][3] * idt : 0.0, cb2 = (O >= 2) ? c_sb[O][2] : 0.0;
  const double ca3 = (O >= 3) ? -c_sa[O][4] * idt : 0.0, cb3 = (O >= 3) ? c_sb[O][3] : 0.0;
#pragma unroll 4
  for (int n = p; n < N; n += 2) {
    const double2 xv = x[n], nv = nn[n];
    E[n] = xv;
    Nn[n] = nv;
    double2 acc = cfma(cb0, nv, cscl(xv, ca0));
    if (O >= 1) acc = cfma(cb1, No0[n], cfma(ca1, Eo0[n], acc));
    if (O >= 2) acc = cfma(cb2, No1[n], cfma(ca2, Eo1[n], acc));
    if (O >= 3) acc = cfma(cb3, No2[n], cfma(ca3, Eo2[n], acc));
    R[n] = acc;
  }
}

__device__ __forceinline__ void lane_sbdf_any(int o, int N, int p, double idt, const double2* x,
                                              const double2* nn, double2* E, double2* Nn,
                                              const double2* const* Eo, const double2* const* No,
                                              double2* R) {
  switch (o) {
    case 0: lane_sbdf<0>(N, p, idt, x, nn, E, Nn, Eo[0], Eo[1], Eo[2], No[0], No[1], No[2], R); break;
    case 1: lane_sbdf<1>(N, p, idt, x, nn, E, Nn, Eo[0], Eo[1], Eo[2], No[0], No[1], No[2], R); break;
    case 2: lane_sbdf<2>(N, p, idt, x, nn, E, Nn, Eo[0], Eo[1], Eo[2], No[0], No[1], No[2], R); break;
    default: lane_sbdf<3>(N, p, idt, x, nn, E, Nn, Eo[0], Eo[1], Eo[2], No[0], No[1], No[2], R); break;
  }
}

// ---------------------------------------------- per-mode spectral stage
// ------------------------------------------------------ Chebyshev columns
// Column transforms along y for a batch of members and fields.  Coefficient
// side: column m, row n at m*cm + n*cn; value side: column m, row j at
// m*vm + j*vj (within one field of one member).  Input and output may be in
// double or single precision independently of the compute type.
constexpr int kYFields = 17;   // columns per launch (blockIdx.y): the 3D inverse pass
struct YJob {
  const void* src;
  void* dst;
  long long src_mstride, dst_mstride;  // per member (elements)
  long long src_fstride, dst_fstride;  // per field (elements)
  int src_field[kYFields];
  int src_field2[kYFields];  // inverse only: >= 0 adds this field to src_field
  int src_field3[kYFields];  // inverse only: >= 0 adds a third field
  int dst_field[kYFields];
  int deriv[kYFields];       // inverse only: transform d/dy of the field
  long long cm, cn;   // coefficient-side strides
  long long vm, vj;   // value-side strides
  int K;              // columns
  int N, M;           // Chebyshev modes, grid intervals / points
  int inverse;        // 1: coefficients -> values; 0: values -> coefficients (N rows)
  int gauss;          // 0: M+1 Gauss-Lobatto points (DCT-I, FFT length 2M);
                      // 1: M Gauss points (DCT-II/III, FFT length M, M even)
  int src_f32, dst_f32;  // element types of src / dst (0: complex double, 1: complex float)
  const double2* tw4;    // gauss: quarter-period table of this direction, k < M:
                         // forward (s_k/2) exp(-i pi k/(2M)) (s_0 = 1/M, s_k = 2/M),
                         // inverse (1/2) exp(+i pi k/(2M))
  const float2* tw4f;    // the same in single precision
  const float4* tw4d;    // the same in double-single (re.h, re.l, im.h, im.l)
  int C;              // columns per block
  const int* status;  // skip members with status != 0 (may be null)
  FftPlan pl;
};

// Element formats of transform inputs and outputs (YJob / ZJob src_f32,
// dst_f32): 0 complex double, 1 complex float, kFmtDS double-single as
// computed (the intermediates of PTT_FP64_DS groups, in their FP64 arrays:
// the same 16 bytes per element).  Only the double-single kernels read or
// write kFmtDS.
constexpr int kFmtDS = 2;
template <typename CT>
__device__ __forceinline__ CT ld2(const void* p, long long i, int f32) {
  if constexpr (std::is_same<CT, dsc>::value) {
    if (f32 == kFmtDS) return static_cast<const dsc*>(p)[i];
  }
  return f32 ? cvt2<CT>(static_cast<const float2*>(p)[i]) : cvt2<CT>(static_cast<const double2*>(p)[i]);
}
template <typename CT>
__device__ __forceinline__ void st2(void* p, long long i, int f32, CT v) {
  if constexpr (std::is_same<CT, dsc>::value) {
    if (f32 == kFmtDS) { static_cast<dsc*>(p)[i] = v; return; }
  }
  if (f32) static_cast<float2*>(p)[i] = cvt2<float2>(v);
  else static_cast<double2*>(p)[i] = cvt2<double2>(v);
}
template <typename CT> __device__ __forceinline__ CT ld_tw4(const YJob& J, int k);
template <> __device__ __forceinline__ double2 ld_tw4<double2>(const YJob& J, int k) { return __ldg(&J.tw4[k]); }
template <> __device__ __forceinline__ float2 ld_tw4<float2>(const YJob& J, int k) { return __ldg(&J.tw4f[k]); }
template <> __device__ __forceinline__ dsc ld_tw4<dsc>(const YJob& J, int k) {
  return ldg_tw(reinterpret_cast<const dsc*>(J.tw4d) + k);
}

// Values at the M Gauss points y_j = cos(pi (2j+1)/(2M)) from coefficients
// (DCT-III) and back (DCT-II), each as one complex FFT of length M: the
// output (input) order is permuted v_n = f_{2n}, v_{M-1-n} = f_{2n+1}, and a
// quarter-period twiddle exp(-+ i pi k/(2M)) maps between the two (Makhoul's
// construction; the real and imaginary parts of a column ride in one FFT).
template <typename CT>
__device__ void ycols_gauss(const YJob& J, const void* src, const void* src2, const void* src3,
                            void* dst, CT* A, CT* B, int c0, int nc, int f) {
  using T = typename RealOf<CT>::T;
  const int C = J.C, N = J.N, Mg = J.M;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (J.inverse) {
    for (int i = tid; i < Mg * C; i += nt) {
      const int c = (int)fdiv((unsigned)i, fast_div((unsigned)Mg)), n = i - c * Mg;
      CT v = zero2<CT>();
      if (c < nc && n < N) {
        const long long o = (c0 + c) * J.cm + n * J.cn;
        v = ld2<CT>(src, o, J.src_f32);
        if (src2) v = cadd(v, ld2<CT>(src2, o, J.src_f32));
        if (src3) v = cadd(v, ld2<CT>(src3, o, J.src_f32));
      }
      A[i] = v;
    }
    __syncthreads();
    if (J.deriv[f]) {
      for (int c = tid >> 5; c < C; c += (nt >> 5)) warp_cheb_deriv(A + c * Mg, B + c * Mg, N);
      __syncthreads();
      for (int i = tid; i < N * C; i += nt) {
        const int c = (int)fdiv((unsigned)i, fast_div((unsigned)N)), n = i - c * N;
        A[c * Mg + n] = B[c * Mg + n];
      }
      __syncthreads();
    }
    // V_0 = a_0, V_k = (1/2) exp(+i pi k/(2M)) (a_k - i a_{M-k}), the factor
    // taken from the inverse table
    for (int i = tid; i < Mg * C; i += nt) {
      const int c = (int)fdiv((unsigned)i, fast_div((unsigned)Mg)), k = i - c * Mg;
      const CT ak = A[i];
      CT V;
      if (k == 0) {
        V = ak;
      } else {
        const CT amk = A[c * Mg + Mg - k];
        CT z;
        z.x = ak.x + amk.y;
        z.y = ak.y - amk.x;
        V = cmul(ld_tw4<CT>(J, k), z);
      }
      B[i] = V;
    }
    __syncthreads();
    CT* res = fft_lines<+1>(B, A, C, Mg, J.pl);
    for (int i = tid; i < Mg * C; i += nt) {
      const int j = (int)fdiv((unsigned)i, fast_div((unsigned)C)), c = i - j * C;
      if (c < nc) {
        const int pos = (j & 1) ? (Mg - 1 - (j >> 1)) : (j >> 1);
        st2<CT>(dst, j * J.vj + (c0 + c) * J.vm, J.dst_f32, res[c * Mg + pos]);
      }
    }
  } else {
    for (int i = tid; i < Mg * C; i += nt) {
      const int j = (int)fdiv((unsigned)i, fast_div((unsigned)C)), c = i - j * C;
      const int pos = (j & 1) ? (Mg - 1 - (j >> 1)) : (j >> 1);
      A[c * Mg + pos] = (c < nc) ? ld2<CT>(src, j * J.vj + (c0 + c) * J.vm, J.src_f32) : zero2<CT>();
    }
    __syncthreads();
    CT* res = fft_lines<-1>(A, B, C, Mg, J.pl);
    // with s = V_k + conj V_{M-k}, d = V_k - conj V_{M-k} (the transforms of
    // the real and imaginary parts, times 2 and 2i) and the forward table
    // F_k = (s_k/2) exp(-i pi k/(2M)):  a_k = (Re(F_k s), Re(F_k (-i d)))
    for (int i = tid; i < N * C; i += nt) {
      const int c = (int)fdiv((unsigned)i, fast_div((unsigned)N)), k = i - c * N;
      if (c < nc) {
        const CT Vk = res[c * Mg + k];
        const CT Rm = res[c * Mg + (k == 0 ? 0 : Mg - k)];
        const T sx = Vk.x + Rm.x, sy = Vk.y - Rm.y;
        const T dx = Vk.x - Rm.x, dy = Vk.y + Rm.y;
        const CT w = ld_tw4<CT>(J, k);
        CT o;
        o.x = w.x * sx - w.y * sy;
        o.y = w.x * dy + w.y * dx;
        st2<CT>(dst, (c0 + c) * J.cm + k * J.cn, J.dst_f32, o);
      }
    }
  }
}

// Gauss-Lobatto path (FP64, or double-single in PTT_FP64_DS groups; FP64
// arrays in and out): DCT-I by the even extension.
template <typename CT>
__device__ void ycols_lobatto(const YJob& J, const void* src, const void* src2, const void* src3,
                              void* dst, CT* A, CT* B, CT* a0s, int c0, int nc, int f) {
  using T = typename RealOf<CT>::T;
  const int C = J.C, N = J.N, M = J.M, P = 2 * J.M;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (J.inverse) {
    for (int i = tid; i < N * C; i += nt) {
      const int c = (int)fdiv((unsigned)i, fast_div((unsigned)N)), n = i - c * N;
      CT v = zero2<CT>();
      if (c < nc) {
        const long long o = (c0 + c) * J.cm + n * J.cn;
        v = ld2<CT>(src, o, 0);
        if (src2) v = cadd(v, ld2<CT>(src2, o, 0));
        if (src3) v = cadd(v, ld2<CT>(src3, o, 0));
      }
      A[c * P + n] = v;
    }
    __syncthreads();
    if (J.deriv[f]) {
      for (int c = tid >> 5; c < C; c += (nt >> 5)) warp_cheb_deriv(A + c * P, B + c * P, N);
      __syncthreads();
      for (int i = tid; i < N * C; i += nt) {
        const int c = (int)fdiv((unsigned)i, fast_div((unsigned)N)), n = i - c * N;
        A[c * P + n] = B[c * P + n];
      }
      __syncthreads();
    }
    if (tid < C) {
      a0s[tid] = A[tid * P];
      a0s[C + tid] = (N > M) ? A[tid * P + M] : zero2<CT>();
    }
    // even extension: A[n] = a_n (n <= M, zero for n >= N), A[P-n] = a_n
    for (int i = tid; i < C * P; i += nt) {
      const int c = (int)fdiv((unsigned)i, fast_div((unsigned)P)), n = i - c * P;
      if (n >= N && n <= M) A[i] = zero2<CT>();
      else if (n > M) { const int r = P - n; A[i] = (r < N) ? A[c * P + r] : zero2<CT>(); }
    }
    __syncthreads();
    CT* res = fft_lines<-1, CT, true>(A, B, C, P, J.pl);
    // f_j = (F_j + a_0 + (-1)^j a_M) / 2
    for (int i = tid; i < (M + 1) * C; i += nt) {
      const int j = (int)fdiv((unsigned)i, fast_div((unsigned)C)), c = i - j * C;
      if (c < nc) {
        CT v = cadd(res[c * P + j], a0s[c]);
        v = (j & 1) ? csub(v, a0s[C + c]) : cadd(v, a0s[C + c]);
        st2<CT>(dst, j * J.vj + (c0 + c) * J.vm, 0, cscl(v, (T)0.5));
      }
    }
  } else {
    for (int i = tid; i < (M + 1) * C; i += nt) {
      const int j = (int)fdiv((unsigned)i, fast_div((unsigned)C)), c = i - j * C;
      A[c * P + j] = (c < nc) ? ld2<CT>(src, j * J.vj + (c0 + c) * J.vm, 0) : zero2<CT>();
    }
    __syncthreads();
    for (int i = tid; i < C * P; i += nt) {
      const int c = (int)fdiv((unsigned)i, fast_div((unsigned)P)), j = i - c * P;
      if (j > M) A[i] = A[c * P + (P - j)];
    }
    __syncthreads();
    CT* res = fft_lines<-1, CT, true>(A, B, C, P, J.pl);
    const T inv = T(1.0 / M);
    for (int i = tid; i < N * C; i += nt) {
      const int c = (int)fdiv((unsigned)i, fast_div((unsigned)N)), n = i - c * N;
      if (c < nc) {
        const T s = (n == 0 || n == M) ? (T)0.5 * inv : inv;
        st2<CT>(dst, (c0 + c) * J.cm + n * J.cn, 0, cscl(res[c * P + n], s));
      }
    }
  }
}

// BIG: the Gauss-Lobatto (unpadded) path, whose FFT length 2 (ny - 1) may
// hold radices 7, 11, 13; the Gauss (padded) path runs without it.
template <typename CT, bool BIG = false>
__device__ __forceinline__ void ycols_block(const YJob& J, Blk bk) {
  const int b = bk.z;
  if (J.status && J.status[b]) return;
  const int f = bk.y;
  // FFT length per column: M on the Gauss grid, 2M (even extension) on the
  // Gauss-Lobatto grid; shared memory holds 2 C lines of it (+ 2 C scalars)
  const int C = J.C, K = J.K, P = J.gauss ? J.M : 2 * J.M;
  const int c0 = bk.x * C;
  const int nc = min(C, K - c0);
  extern __shared__ __align__(16) unsigned char smraw[];
  CT* A = reinterpret_cast<CT*>(smraw);
  CT* B = A + (size_t)C * P;
  const size_t es = (J.src_f32 == 1) ? sizeof(float2) : sizeof(double2);
  const size_t ed = (J.dst_f32 == 1) ? sizeof(float2) : sizeof(double2);
  const void* src = static_cast<const char*>(J.src) + (b * J.src_mstride + J.src_field[f] * J.src_fstride) * es;
  void* dst = static_cast<char*>(J.dst) + (b * J.dst_mstride + J.dst_field[f] * J.dst_fstride) * ed;
  const void* src2 = (J.inverse && J.src_field2[f] >= 0)
      ? static_cast<const char*>(J.src) + (b * J.src_mstride + J.src_field2[f] * J.src_fstride) * es
      : nullptr;
  const void* src3 = (J.inverse && J.src_field3[f] >= 0)
      ? static_cast<const char*>(J.src) + (b * J.src_mstride + J.src_field3[f] * J.src_fstride) * es
      : nullptr;
  if (J.gauss) {
    ycols_gauss<CT>(J, src, src2, src3, dst, A, B, c0, nc, f);
  } else if constexpr (!std::is_same<CT, float2>::value && BIG) {
    ycols_lobatto<CT>(J, src, src2, src3, dst, A, B, B + (size_t)C * P, c0, nc, f);
  }
}

template <typename CT, bool BIG = false>
__global__ void __launch_bounds__(256) k_ycols(YJob J) {
  ycols_block<CT, BIG>(J, this_blk());
}

// The same over the shape groups of a context (job q of jobs for group q).
template <typename CT, bool BIG = false>
__global__ void __launch_bounds__(256) k_ycols_multi(const YJob* __restrict__ jobs, MultiMap mm) {
  Blk bk;
  const int q = multi_locate(mm, bk);
  ycols_block<CT, BIG>(jobs[q], bk);
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
  int nf;                    // fields (packed in pairs, (nf + 1) / 2 lines)
  int K, n;
  int c2r;
  // c2r with nf = 1: block r synthesises rows 2r and 2r + 1 (< nrows) as the
  // real and imaginary parts of one line (grid over ceil(nrows / 2) rows)
  int pair_rows, nrows;
  const int* status;
  FftPlan pl;
};

__device__ __forceinline__ void xrows_block(const XJob& J, Blk bk) {
  const int b = bk.y;
  if (J.status && J.status[b]) return;
  const int row = bk.x;
  const int K = J.K, n = J.n, nf = J.nf, nl = (nf + 1) / 2;
  extern __shared__ double2 sm[];
  double2* A = sm;
  double2* Bb = sm + (size_t)nl * n;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (J.c2r) {
    // paired rows: the second line's source and destination are the next row
    const bool pr = J.pair_rows != 0;
    const int r0 = pr ? 2 * row : row;
    const int nfe = pr ? ((r0 + 1 < J.nrows) ? 2 : 1) : nf;
    const long long sfs = pr ? (long long)J.src_rstep * K : J.src_fstride;
    const long long dfs = pr ? (long long)J.dst_rstep * n : J.dst_fstride;
    const double2* src = J.srcC + b * J.src_mstride + (long long)r0 * J.src_rstep * K;
    for (int i = tid; i < nl * n; i += nt) {
      const int l = (int)fdiv((unsigned)i, fast_div((unsigned)n)), k = i - l * n;
      const int fa = 2 * l, fb = 2 * l + 1;
      int kk = -1;
      bool cj = false;
      if (k < K) kk = k;
      else if (k > n - K) { kk = n - k; cj = true; }
      double2 h = czero();
      if (kk >= 0) {
        double2 F = src[fa * sfs + kk];
        double2 G = (fb < nfe) ? src[fb * sfs + kk] : czero();
        if (kk == 0) { F.y = 0.0; G.y = 0.0; }
        if (cj) { F = cconj(F); G = cconj(G); }
        h = cadd(F, mul_i(G));
      }
      A[i] = h;
    }
    __syncthreads();
    double2* res = fft_lines<+1, double2, true>(A, Bb, nl, n, J.pl);
    double* dst = J.dstR + b * J.dst_mstride + (long long)r0 * J.dst_rstep * n;
    for (int i = tid; i < nl * n; i += nt) {
      const int l = (int)fdiv((unsigned)i, fast_div((unsigned)n)), x = i - l * n;
      const double2 h = res[i];
      dst[(2 * l) * dfs + x] = h.x;
      if (2 * l + 1 < nfe) dst[(2 * l + 1) * dfs + x] = h.y;
    }
  } else {
    const double* src = J.srcR + b * J.src_mstride + (long long)row * J.src_rstep * n;
    for (int i = tid; i < nl * n; i += nt) {
      const int l = (int)fdiv((unsigned)i, fast_div((unsigned)n)), x = i - l * n;
      const double fa = src[(2 * l) * J.src_fstride + x];
      const double fb = (2 * l + 1 < nf) ? src[(2 * l + 1) * J.src_fstride + x] : 0.0;
      A[i] = make_double2(fa, fb);
    }
    __syncthreads();
    double2* res = fft_lines<-1, double2, true>(A, Bb, nl, n, J.pl);
    double2* dst = J.dstC + b * J.dst_mstride + (long long)row * J.dst_rstep * K;
    const double inv = 1.0 / n;
    for (int i = tid; i < nl * K; i += nt) {
      const int l = (int)fdiv((unsigned)i, fast_div((unsigned)K)), k = i - l * K;
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


__global__ void __launch_bounds__(256) k_xrows(XJob J) { xrows_block(J, this_blk()); }

__global__ void __launch_bounds__(256) k_xrows_multi(const XJob* __restrict__ jobs, MultiMap mm) {
  Blk bk;
  const int q = multi_locate(mm, bk);
  xrows_block(jobs[q], bk);
}


// ------------------------------------------------------------ reductions
// The diagnostics compare, bound and count doubles through order-preserving
// integer keys: FP64 compares, min/max and additions run at the FP64 rate
// (about 1/64 of the FP32 rate here), integer ones at the ALU rate.
// key(x) < key(y) exactly when x < y, for x, y not NaN, except -0 < +0.
__device__ __forceinline__ long long dkey(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double dkey_val(long long k) {   // inverse of dkey
  return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}
__device__ __forceinline__ bool isnan_bits(double x) {
  return (__double_as_longlong(x) & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL;
}

// Extrema of Tr c as keys (min, max) and |Tr c| as bits (a non-negative
// double orders as its bit pattern); NaN values are left out, as fmin and
// fmax leave them out.  Empty: min LLONG_MAX, max LLONG_MIN, amax 0.
struct KeyExt {
  long long mn, mx, ma;
};
__device__ __forceinline__ KeyExt keyext_empty() {
  return KeyExt{0x7fffffffffffffffLL, (long long)0x8000000000000000ULL, 0LL};
}
__device__ __forceinline__ void keyext_add(KeyExt& e, double t) {
  if (isnan_bits(t)) return;
  const long long k = dkey(t);
  e.mn = min(e.mn, k);
  e.mx = max(e.mx, k);
  e.ma = max(e.ma, __double_as_longlong(t) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ void keyext_merge(KeyExt& e, const KeyExt& o) {
  e.mn = min(e.mn, o.mn);
  e.mx = max(e.mx, o.mx);
  e.ma = max(e.ma, o.ma);
}
__device__ __forceinline__ KeyExt keyext_shfl_down(const KeyExt& e, int o) {
  return KeyExt{__shfl_down_sync(0xffffffffu, e.mn, o), __shfl_down_sync(0xffffffffu, e.mx, o),
                __shfl_down_sync(0xffffffffu, e.ma, o)};
}

// The counts of t < 3, t < 0, |t - 3| <= tau and |t| <= tau on keys.  For
// tau <= 1.5, t - 3 is exact wherever |t - 3| <= tau can hold (Sterbenz's
// lemma), so the band is the closed interval [RU(3 - tau), RD(3 + tau)] of
// doubles; |t| <= tau is [-tau, tau] exactly.  A larger tau (a field far
// past any physical value) takes the FP64 test.  NaN counts nowhere, as in
// the FP64 comparisons.
struct TrBands {
  long long k3, lo3, hi3, lo0, hi0;
  double tau;
  bool exact;
};
__device__ __forceinline__ TrBands tr_bands(double tau) {
  TrBands B;
  B.tau = tau;
  B.exact = (tau <= 1.5);
  B.k3 = dkey(3.0);
  B.lo3 = dkey(__dsub_ru(3.0, tau));
  B.hi3 = dkey(__dadd_rd(3.0, tau));
  B.lo0 = dkey(-tau);
  B.hi0 = dkey(tau);
  return B;
}
struct TrCounts {
  int c3, c0, b3, b0;
};
__device__ __forceinline__ void tr_count(TrCounts& c, double t, const TrBands& B) {
  if (isnan_bits(t)) return;
  const long long k = dkey(t);
  c.c3 += (k < B.k3);
  c.c0 += (k < -1LL);   // below key(-0.0) = -1: negative and nonzero
  if (B.exact) {
    c.b3 += (k >= B.lo3 && k <= B.hi3);
    c.b0 += (k >= B.lo0 && k <= B.hi0);
  } else {
    c.b3 += (fabs(t - 3.0) <= B.tau);
    c.b0 += (fabs(t) <= B.tau);
  }
}

// Block-wide sums of 64-bit integers and merges of extrema (fixed order).
// sh: shared memory of at least 3 * 32 long longs; the results are valid in
// every thread.
__device__ long long block_isum(long long v, long long* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  long long s = 0;
  for (int i = 0; i < nw; ++i) s += sh[i];
  __syncthreads();
  return s;
}
__device__ KeyExt block_keyext(KeyExt e, long long* sh) {
  for (int o = 16; o > 0; o >>= 1) keyext_merge(e, keyext_shfl_down(e, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) { sh[w] = e.mn; sh[32 + w] = e.mx; sh[64 + w] = e.ma; }
  __syncthreads();
  KeyExt r = keyext_empty();
  for (int i = 0; i < nw; ++i) keyext_merge(r, KeyExt{sh[i], sh[32 + i], sh[64 + i]});
  __syncthreads();
  return r;
}

// Sums of 32 per-thread values over the block, one total per value: a
// reduce-scatter across the lanes (at each of five levels a lane keeps half
// of its values and adds its partner's copies of them: 31 additions per
// lane, against 5 per value for a tree per value), then across the warps in
// index order.  v is consumed; on return red[k], k < 32, holds the total of
// v[k] (a fixed order: deterministic).  red: 32 * (blockDim.x / 32) doubles
// of shared memory.
__device__ void block_sum_scatter(double (&v)[32], double* red) {
  const int l = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool up = (l & s) != 0;
#pragma unroll
    for (int i = 0; i < s; ++i) {
      const double send = up ? v[i] : v[i + s];
      const double keep = up ? v[i + s] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  // lane l holds its warp's total of value l (index bits kept level by level)
  __syncthreads();
  red[w * 32 + l] = v[0];
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = red[threadIdx.x];
    for (int i = 1; i < nw; ++i) t += red[i * 32 + threadIdx.x];
    red[threadIdx.x] = t;
  }
  __syncthreads();
}

// Max of the non-negative doubles stored as bits in pp[t * kPart + slot]
// over the ntile tiles of one member, on their bit patterns; every thread of
// the block receives it.
__device__ double block_tiles_amax(const double* pp, int ntile, int slot) {
  __shared__ long long smk[32];
  const long long* q = reinterpret_cast<const long long*>(pp);
  long long m = 0;
  for (int t = threadIdx.x; t < ntile; t += blockDim.x) m = max(m, q[(size_t)t * kPart + slot]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) smk[w] = m;
  __syncthreads();
  for (int i = 0; i < nw; ++i) m = max(m, smk[i]);
  __syncthreads();
  return __longlong_as_double(m);
}

// Max of pp[t * kPart + slot] over the ntile tiles of one member; every
// thread of the block receives it.
__device__ double block_tiles_max(const double* pp, int ntile, int slot) {
  __shared__ double sm[32];
  double m = 0.0;
  for (int t = threadIdx.x; t < ntile; t += blockDim.x) m = fmax(m, pp[(size_t)t * kPart + slot]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sm[w] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) m = fmax(m, sm[i]);
    sm[0] = m;
  }
  __syncthreads();
  const double r = sm[0];
  __syncthreads();
  return r;
}

// Block sums of NV values at once (fixed order: lanes by shuffles, then
// warps in index order).  red: shared memory of (blockDim.x / 32) * NV
// doubles; on return red[k], k < NV, holds the sum of v[k] over the block.
template <int NV>
__device__ void block_sum_many(const double (&v)[NV], double* red) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = v[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (l == 0) red[w * NV + k] = x;
  }
  __syncthreads();
  double sum = 0.0;
  if (threadIdx.x < NV)
    for (int i = 0; i < nw; ++i) sum += red[i * NV + threadIdx.x];
  __syncthreads();
  if (threadIdx.x < NV) red[threadIdx.x] = sum;
  __syncthreads();
}

// Histogram slot of x for the range [lo, hi) (PTT_HIST_BINS uniform bins,
// slot 0 below lo, slot PTT_HIST_BINS + 1 at or above hi or not finite);
// -1 when the quantity is switched off (lo >= hi).
__device__ __forceinline__ int hist_slot(double x, double lo, double hi) {
  if (!(lo < hi)) return -1;
  if (!isfinite(x) || x >= hi) return PTT_HIST_BINS + 1;
  if (x < lo) return 0;
  const int k = (int)floor((x - lo) * ((double)PTT_HIST_BINS / (hi - lo)));
  return 1 + min(k, PTT_HIST_BINS - 1);
}

// Block-wide max of v (fixed order), valid in thread 0.
__device__ double block_tiles_max_val(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) v = fmax(v, sh[i]);
  return v;
}

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


inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

}  // namespace
}  // namespace ptt
