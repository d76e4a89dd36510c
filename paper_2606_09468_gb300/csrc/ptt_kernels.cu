// Device code of the FP64 pseudo-spectral sPTT channel step (2D, sm_103a).
//
// One step (Sec. 2: fully dealiased Fourier-Chebyshev pseudo-spectral method,
// fourth-order semi-implicit BDF) is the launch sequence
//   k_ycols  (inverse)  spectral (m, n) -> values on the padded Gauss-Lobatto
//                       y grid, with d/dy by the Chebyshev recurrence
//   k_xfused            per padded y row: inverse x FFTs of 14 fields, the
//                       sPTT / advection products of Eqs. 1-2, forward x FFTs
//   k_ycols  (forward)  padded y values -> Chebyshev coefficients (truncated)
//   k_rhs               linear explicit terms, curl-curl forcing, SBDF sums
//   k_solve             per (mode, system, parity) quasi-tridiagonal tau solve
//   k_uvel              u from continuity, step counter
// followed by the diagnostics of Sec. 3 (k_ycols, k_diag_part, k_xrows,
// k_diag_final).  All transforms are mixed-radix (2, 3, 4, 5) Stockham FFTs
// in shared memory; the Chebyshev transforms are discrete cosine transforms
// of type I computed as FFTs of the even extension.
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

// ------------------------------------------------------------ radix DFTs
// DIR = -1: exp(-2 pi i jk/R) (forward); DIR = +1: exp(+2 pi i jk/R).
template <int DIR, int R> struct Bfly;

template <int DIR> struct Bfly<DIR, 2> {
  static __device__ __forceinline__ void run(double2* v) {
    double2 t = v[0];
    v[0] = cadd(t, v[1]);
    v[1] = csub(t, v[1]);
  }
};

template <int DIR> struct Bfly<DIR, 4> {
  static __device__ __forceinline__ void run(double2* v) {
    double2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    double2 s13 = cadd(v[1], v[3]), d13 = mul_i(csub(v[1], v[3]));
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    if (DIR < 0) { v[1] = csub(d02, d13); v[3] = cadd(d02, d13); }
    else         { v[1] = cadd(d02, d13); v[3] = csub(d02, d13); }
  }
};

template <int DIR> struct Bfly<DIR, 3> {
  static __device__ __forceinline__ void run(double2* v) {
    const double s = DIR * 0.86602540378443864676;  // sin(2 pi / 3), signed
    double2 t1 = cadd(v[1], v[2]);
    double2 it2 = mul_i(csub(v[1], v[2]));
    double2 m = cfma(-0.5, t1, v[0]);
    v[0] = cadd(v[0], t1);
    v[1] = cfma(s, it2, m);
    v[2] = cfma(-s, it2, m);
  }
};

template <int DIR> struct Bfly<DIR, 5> {
  static __device__ __forceinline__ void run(double2* v) {
    const double c1 = 0.30901699437494742410;   // cos(2 pi / 5)
    const double c2 = -0.80901699437494742410;  // cos(4 pi / 5)
    const double s1 = DIR * 0.95105651629515357212;  // sin(2 pi / 5), signed
    const double s2 = DIR * 0.58778525229247312917;  // sin(4 pi / 5), signed
    double2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    double2 t3 = mul_i(csub(v[1], v[4])), t4 = mul_i(csub(v[2], v[3]));
    double2 b1 = cfma(c1, t1, cfma(c2, t2, v[0]));
    double2 b2 = cfma(c2, t1, cfma(c1, t2, v[0]));
    double2 e1 = cfma(s1, t3, cscl(t4, s2));
    double2 e2 = cfma(s2, t3, cscl(t4, -s1));
    v[0] = cadd(v[0], cadd(t1, t2));
    v[1] = cadd(b1, e1);
    v[4] = csub(b1, e1);
    v[2] = cadd(b2, e2);
    v[3] = csub(b2, e2);
  }
};

// One Stockham pass of radix R over nl lines (line l at offset l*ls).
template <int DIR, int R>
__device__ __forceinline__ void fft_pass(const double2* __restrict__ src, double2* __restrict__ dst,
                                         int nl, int ls, int n, int Ns,
                                         const double2* __restrict__ tw) {
  const int nb = n / R;
  const int st = n / (Ns * R);
  const int total = nl * nb;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int l = t / nb;
    const int j = t - l * nb;
    const double2* s = src + l * ls;
    double2* d = dst + l * ls;
    const int jm = j % Ns;
    double2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = s[j + r * nb];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        double2 w = __ldg(&tw[jm * r * st]);
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

// Unnormalised DFT of nl lines of length pl.n held in `a`, using `b` as the
// ping-pong buffer.  Returns the buffer holding the result.  Must be called
// by the whole block after a __syncthreads(); ends with one.
template <int DIR>
__device__ double2* fft_lines(double2* a, double2* b, int nl, int ls, const FftPlan& pl) {
  double2* src = a;
  double2* dst = b;
  int Ns = 1;
  for (int s = 0; s < pl.nst; ++s) {
    const int R = pl.radix[s];
    switch (R) {
      case 2: fft_pass<DIR, 2>(src, dst, nl, ls, pl.n, Ns, pl.tw); break;
      case 3: fft_pass<DIR, 3>(src, dst, nl, ls, pl.n, Ns, pl.tw); break;
      case 4: fft_pass<DIR, 4>(src, dst, nl, ls, pl.n, Ns, pl.tw); break;
      default: fft_pass<DIR, 5>(src, dst, nl, ls, pl.n, Ns, pl.tw); break;
    }
    __syncthreads();
    Ns *= R;
    double2* t = src; src = dst; dst = t;
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

// ------------------------------------------------------ Chebyshev columns
// Column transforms along y for a batch of members and fields.
struct YJob {
  const double2* src;
  double2* dst;
  long long src_mstride, dst_mstride;  // per member (elements)
  long long src_fstride, dst_fstride;  // per field (elements)
  int src_field[8];
  int dst_field[8];
  int deriv[8];       // inverse only: transform d/dy of the field
  int K;              // columns (= row length)
  int N, M;           // Chebyshev modes, grid intervals (P = 2M)
  int inverse;        // 1: coefficients -> values (M+1 rows); 0: values -> coefficients (N rows)
  int C;              // columns per block
  const int* status;  // skip members with status != 0 (may be null)
  FftPlan pl;
};

// Chebyshev derivative in place: b_{n-1} = b_{n+1} + 2 n a_n, b_0 halved.
__device__ void cheb_deriv_inplace(double2* a, int N) {
  double2 bnp1 = czero(), bn = czero();
  double2 acur = a[N - 1];
  a[N - 1] = czero();
  for (int n = N - 1; n >= 1; --n) {
    double2 anext = a[n - 1];
    double2 bnm1 = cfma(2.0 * n, acur, bnp1);
    a[n - 1] = bnm1;
    bnp1 = bn;
    bn = bnm1;
    acur = anext;
  }
  a[0] = cscl(a[0], 0.5);
}

__global__ void __launch_bounds__(256) k_ycols(YJob J) {
  const int b = blockIdx.z;
  if (J.status && J.status[b]) return;
  const int f = blockIdx.y;
  const int C = J.C, K = J.K, N = J.N, M = J.M, P = 2 * J.M;
  const int c0 = blockIdx.x * C;
  const int nc = min(C, K - c0);
  extern __shared__ double2 sm[];
  double2* A = sm;
  double2* B = sm + (size_t)C * P;
  double2* a0s = B + (size_t)C * P;  // [C] a_0, [C] a_M
  const double2* src = J.src + b * J.src_mstride + J.src_field[f] * J.src_fstride + c0;
  double2* dst = J.dst + b * J.dst_mstride + J.dst_field[f] * J.dst_fstride + c0;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (J.inverse) {
    for (int i = tid; i < N * C; i += nt) {
      const int n = i / C, c = i - n * C;
      A[c * P + n] = (c < nc) ? src[(size_t)n * K + c] : czero();
    }
    __syncthreads();
    if (J.deriv[f]) {
      if (tid < C) cheb_deriv_inplace(A + tid * P, N);
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
        dst[(size_t)j * K + c] = cscl(v, 0.5);
      }
    }
  } else {
    for (int i = tid; i < (M + 1) * C; i += nt) {
      const int j = i / C, c = i - j * C;
      A[c * P + j] = (c < nc) ? src[(size_t)j * K + c] : czero();
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
      const int n = i / C, c = i - n * C;
      if (c < nc) {
        const double s = (n == 0 || n == M) ? 0.5 * inv : inv;
        dst[(size_t)n * K + c] = cscl(res[c * P + n], s);
      }
    }
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

__global__ void __launch_bounds__(512) k_xfused(GroupDev g) {
  const int b = blockIdx.y;
  if (g.status[b]) return;
  const int j = blockIdx.x;
  const int K = g.K, Mx = g.Mx, rows = g.M + 1;
  const MemberPrm pr = g.prm[b];
  extern __shared__ double2 sm[];
  double2* A = sm;
  double2* B = sm + 7 * Mx;
  const double2* Y = g.Yp + (size_t)b * 9 * rows * K + (size_t)j * K;
  const double kfac = 2.0 * 3.14159265358979323846 / pr.lx;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < 7 * Mx; i += nt) {
    const int l = i / Mx, k = i - l * Mx;
    int kk = -1;
    bool cj = false;
    if (k < K) kk = k;
    else if (k > Mx - K) { kk = Mx - k; cj = true; }
    double2 h = czero();
    if (kk >= 0) {
      const int fa = 2 * l, fb = 2 * l + 1;
      double2 F = Y[(size_t)c_xsrc[fa] * rows * K + kk];
      double2 G = Y[(size_t)c_xsrc[fb] * rows * K + kk];
      if (kk == 0) { F.y = 0.0; G.y = 0.0; }
      const double km = kfac * kk;
      if (c_xik[fa]) F = cscl(mul_i(F), km);
      if (c_xik[fb]) G = cscl(mul_i(G), km);
      if (cj) { F = cconj(F); G = cconj(G); }
      h = cadd(F, mul_i(G));
    }
    A[i] = h;
  }
  __syncthreads();
  double2* res = fft_lines<+1>(A, B, 7, Mx, g.plMx);
  double2* oth = (res == A) ? B : A;
  const double eps = pr.eps, iwi = pr.inv_wi;
  for (int x = tid; x < Mx; x += nt) {
    const double2 h0 = res[x], h1 = res[Mx + x], h2 = res[2 * Mx + x], h3 = res[3 * Mx + x];
    const double2 h4 = res[4 * Mx + x], h5 = res[5 * Mx + x], h6 = res[6 * Mx + x];
    const double u = h0.x, v = h0.y, uy = h1.x, ux = h1.y, vx = h2.x, cxx = h2.y;
    const double cxy = h3.x, cyy = h3.y, cxx_y = h4.x, cxy_y = h4.y, cyy_y = h5.x;
    const double cxx_x = h5.y, cxy_x = h6.x, cyy_x = h6.y;
    // Eq. 1: L_ij = du_i/dx_j (L_yy = -ux by continuity); relaxation factor
    // f = 1 + eps Tr(c - I) with c_zz = 1.
    const double rw = (1.0 + eps * (cxx + cyy - 2.0)) * iwi;
    const double ncxx = -(u * cxx_x + v * cxx_y) + 2.0 * (ux * cxx + uy * cxy) - (cxx - 1.0) * rw;
    const double ncxy = -(u * cxy_x + v * cxy_y) + uy * cyy + vx * cxx - cxy * rw;
    const double ncyy = -(u * cyy_x + v * cyy_y) + 2.0 * (vx * cxy - ux * cyy) - (cyy - 1.0) * rw;
    // Eq. 2 advection
    const double nu_ = -(u * ux + v * uy);
    const double nv_ = -(u * vx - v * ux);
    oth[x] = make_double2(ncxx, ncxy);
    oth[Mx + x] = make_double2(ncyy, nu_);
    oth[2 * Mx + x] = make_double2(nv_, 0.0);
  }
  __syncthreads();
  double2* r2 = fft_lines<-1>(oth, res, 3, Mx, g.plMx);
  double2* Z = g.Zp + (size_t)b * 5 * rows * K + (size_t)j * K;
  const double inv = 1.0 / Mx;
  for (int i = tid; i < 3 * K; i += nt) {
    const int l = i / K, k = i - l * K;
    const double2 hk = r2[l * Mx + k];
    const double2 hm = cconj(r2[l * Mx + (k == 0 ? 0 : Mx - k)]);
    const double2 F = cscl(cadd(hk, hm), 0.5 * inv);
    const double2 d = csub(hk, hm);
    const double2 G = make_double2(0.5 * inv * d.y, -0.5 * inv * d.x);
    Z[(size_t)(2 * l) * rows * K + k] = F;
    if (l < 2) Z[(size_t)(2 * l + 1) * rows * K + k] = G;
  }
}

// ------------------------------------------------ explicit terms and SBDF
// One thread per (member, Fourier mode m); loops over the Chebyshev index.
// NR fields: 0 Ncxx, 1 Ncxy, 2 Ncyy, 3 Nu (advection), 4 Nv.
// mode 0: full step; mode 1: only H_x, H_y into Rb[0], Rb[1] (no history).
__global__ void k_rhs(GroupDev g, int mode) {
  const int b = blockIdx.y;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= g.K || g.status[b]) return;
  const int K = g.K, N = g.N, nb = g.nb;
  const size_t NK = (size_t)N * K;
  const MemberPrm pr = g.prm[b];
  const long long cnt = g.count[b];
  const int slot = (int)(cnt & 3);
  const double km = 2.0 * 3.14159265358979323846 * m / pr.lx;
  const double km2 = km * km;
  const double gam = pr.gam;
  const double2* X = g.X + (size_t)b * 5 * NK + m;
  const double2* NR = g.NR + (size_t)b * 5 * NK + m;
  double2* R = g.Rb + (size_t)b * 4 * NK + m;
  // pass 1: H_x = Nu + gam (i k cxx + D cxy) (+ 2/Re on the mean mode),
  //         H_y = Nv + gam (i k cxy + D cyy)                        (Eq. 2)
  {
    double2 p1 = czero(), p0 = czero(), q1 = czero(), q0 = czero();
    double2 axy = X[3 * NK + (size_t)(N - 1) * K], ayy = X[4 * NK + (size_t)(N - 1) * K];
    for (int n = N - 1; n >= 0; --n) {
      const double2 dxy = (n == 0) ? cscl(p0, 0.5) : p0;
      const double2 dyy = (n == 0) ? cscl(q0, 0.5) : q0;
      const size_t o = (size_t)n * K;
      const double2 cxx = X[2 * NK + o], cxy = axy, cyy = ayy;
      double2 hx = cadd(NR[3 * NK + o], cscl(cadd(cscl(mul_i(cxx), km), dxy), gam));
      double2 hy = cadd(NR[4 * NK + o], cscl(cadd(cscl(mul_i(cxy), km), dyy), gam));
      if (m == 0 && n == 0) hx.x += pr.forcing;
      R[0 * NK + o] = hx;
      R[1 * NK + o] = hy;
      if (n >= 1) {
        const double2 nxy = X[3 * NK + o - K], nyy = X[4 * NK + o - K];
        const double2 pm = cfma(2.0 * n, cxy, p1);
        const double2 qm = cfma(2.0 * n, cyy, q1);
        p1 = p0; p0 = pm; q1 = q0; q0 = qm;
        axy = nxy; ayy = nyy;
      }
    }
  }
  if (mode == 1) return;
  double2* E = g.Eh + ((size_t)slot * nb + b) * 4 * NK + m;
  double2* Nn = g.Nh + ((size_t)slot * nb + b) * 4 * NK + m;
  // pass 2: forcing of the evolved velocity quantity.  m >= 1: the curl of
  // Eq. 2 taken twice, -D(i k H_x) - k^2 H_y; m = 0: H_x (mean flow).
  {
    double2 p1 = czero(), p0 = czero();
    double2 ahx = R[(size_t)(N - 1) * K];
    for (int n = N - 1; n >= 0; --n) {
      const size_t o = (size_t)n * K;
      const double2 dhx = (n == 0) ? cscl(p0, 0.5) : p0;
      const double2 hx = ahx;
      double2 nq;
      if (m == 0) nq = hx;
      else nq = csub(cscl(mul_i(dhx), -km), cscl(R[1 * NK + o], km2));
      Nn[3 * NK + o] = nq;
      Nn[0 * NK + o] = NR[0 * NK + o];
      Nn[1 * NK + o] = NR[1 * NK + o];
      Nn[2 * NK + o] = NR[2 * NK + o];
      E[0 * NK + o] = X[2 * NK + o];
      E[1 * NK + o] = X[3 * NK + o];
      E[2 * NK + o] = X[4 * NK + o];
      if (n >= 1) {
        const double2 nhx = R[o - K];
        const double2 pm = cfma(2.0 * n, hx, p1);
        p1 = p0; p0 = pm;
        ahx = nhx;
      }
    }
  }
  // pass 3: evolved velocity quantity q = (D^2 - k^2) v (m >= 1), U (m = 0)
  if (m == 0) {
    for (int n = 0; n < N; ++n) E[3 * NK + (size_t)n * K] = X[(size_t)n * K];
  } else {
    // D v into R[2]
    double2 p1 = czero(), p0 = czero();
    double2 av = X[1 * NK + (size_t)(N - 1) * K];
    for (int n = N - 1; n >= 0; --n) {
      const size_t o = (size_t)n * K;
      R[2 * NK + o] = (n == 0) ? cscl(p0, 0.5) : p0;
      if (n >= 1) {
        const double2 nv = X[1 * NK + o - K];
        const double2 pm = cfma(2.0 * n, av, p1);
        p1 = p0; p0 = pm; av = nv;
      }
    }
    p1 = czero(); p0 = czero();
    double2 ad = R[2 * NK + (size_t)(N - 1) * K];
    for (int n = N - 1; n >= 0; --n) {
      const size_t o = (size_t)n * K;
      const double2 d2 = (n == 0) ? cscl(p0, 0.5) : p0;
      E[3 * NK + o] = cfma(-km2, X[1 * NK + o], d2);
      if (n >= 1) {
        const double2 nd = R[2 * NK + o - K];
        const double2 pm = cfma(2.0 * n, ad, p1);
        p1 = p0; p0 = pm; ad = nd;
      }
    }
  }
  // pass 4: SBDF right-hand sides R_s = sum_j (-a_{j+1}/dt) x^{n-j}_s + b_j N^{n-j}_s
  const int o4 = (cnt < 3) ? (int)cnt : 3;
  const double idt = 1.0 / pr.dt;
  for (int s = 0; s < 4; ++s) {
    for (int n = 0; n < N; ++n) {
      const size_t o = (size_t)s * NK + (size_t)n * K;
      double2 acc = czero();
      for (int jj = 0; jj <= o4; ++jj) {
        const size_t sl = (size_t)((slot - jj) & 3);
        const double2 ex = g.Eh[(sl * nb + b) * 4 * NK + m + o];
        const double2 en = g.Nh[(sl * nb + b) * 4 * NK + m + o];
        acc = cfma(-c_sa[o4][jj + 1] * idt, ex, acc);
        acc = cfma(c_sb[o4][jj], en, acc);
      }
      R[o] = acc;
    }
  }
}

// Quasi-tridiagonal Chebyshev-tau solve of one parity p of
//   (alpha - beta D^2) a = rsign * R   on tau rows n <= N-3,
//   sum_{n = p mod 2} a_n = bcfac * sum_{n = p mod 2} rsign * R_n.
// Rows n >= 2 of the system in the form obtained by integrating twice
// (three-term in n; the operator tables Q, inv, F and G carry the
// right-hand-side-independent part of the elimination).  `out` may alias R.
__device__ void qt_solve(int N, int K, int p, double alpha, const double2* R, double2* out,
                         const double* Q, const double* inv, const double* F, double G,
                         const double* w1, const double* w2, const double* w3,
                         double bcfac, double rsign) {
  const int nl = ((N - 1 - p) & ~1) + p;
  double2 Pn2 = czero(), U = czero(), rsum = czero();
  double2 Rp2 = czero();
  double2 R0 = cscl(R[(size_t)nl * K], rsign);
  for (int n = nl; n >= p + 2; n -= 2) {
    const double2 Rm2 = cscl(R[(size_t)(n - 2) * K], rsign);
    rsum = cadd(rsum, R0);
    const double c = (n == 2) ? 2.0 : 1.0;
    double2 r = cscl(Rm2, -c * w1[n]);
    if (n <= N - 3) r = cfma(w2[n], R0, r);
    double un = 0.0;
    if (n <= N - 5) { r = cfma(-w3[n], Rp2, r); un = -alpha * w3[n]; }
    const double2 P = cscl(cfma(-un, Pn2, r), inv[(size_t)n * K]);
    out[(size_t)n * K] = P;
    U = cfma(F[(size_t)n * K], P, U);
    Pn2 = P;
    Rp2 = R0;
    R0 = Rm2;
  }
  rsum = cadd(rsum, R0);
  double2 a = cscl(csub(cscl(rsum, bcfac), U), G);
  out[(size_t)p * K] = a;
  for (int n = p + 2; n <= nl; n += 2) {
    a = cfma(Q[(size_t)n * K], a, out[(size_t)n * K]);
    out[(size_t)n * K] = a;
  }
}

// One thread per (member, mode m, system, parity).  Systems: 0-2 the c
// components (Helmholtz with the wall-ODE Dirichlet rows), 3 the velocity
// (m = 0: mean-flow Helmholtz; m >= 1: v-phi by the influence matrix).
__global__ void k_solve(GroupDev g) {
  const int b = blockIdx.z;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= g.K || g.status[b]) return;
  const int sys = blockIdx.y >> 1, p = blockIdx.y & 1;
  const int K = g.K, N = g.N;
  const size_t NK = (size_t)N * K;
  const MemberPrm pr = g.prm[b];
  const long long cnt = g.count[b];
  const int o = (cnt < 3) ? (int)cnt : 3;
  const double a0 = c_sa[o][0];
  const double km = 2.0 * 3.14159265358979323846 * m / pr.lx;
  const double km2 = km * km;
  double2* X = g.X + (size_t)b * 5 * NK + m;
  double2* R = g.Rb + (size_t)b * 4 * NK + (size_t)sys * NK + m;
  const double* w1 = g.wrow;
  const double* w2 = g.wrow + N;
  const double* w3 = g.wrow + 2 * N;
  auto tab = [&](int ts, int which) {
    return g.qt + (((((size_t)b * 4 + o) * 3 + ts) * 3 + which) * NK) + m;
  };
  auto tabG = [&](int ts) { return g.qtG[((((size_t)b * 4 + o) * 3 + ts) * 2 + p) * K + m]; };
  if (sys < 3) {
    double2* out = X + (size_t)(2 + sys) * NK;
    const double alpha = a0 / pr.dt + pr.kappa * km2;
    if (pr.kappa == 0.0) {
      const double ia = 1.0 / alpha;
      for (int n = p; n < N; n += 2) out[(size_t)n * K] = cscl(R[(size_t)n * K], ia);
      return;
    }
    qt_solve(N, K, p, alpha, R, out, tab(0, 0), tab(0, 1), tab(0, 2), tabG(0), w1, w2, w3,
             pr.dt / a0, 1.0);
    return;
  }
  if (m == 0) {
    qt_solve(N, K, p, a0 / pr.dt, R, X, tab(1, 0), tab(1, 1), tab(1, 2), tabG(1), w1, w2, w3,
             0.0, 1.0);
    for (int n = p; n < N; n += 2) X[NK + (size_t)n * K] = czero();
    return;
  }
  // phi_p (in place in R), then v_p, then the influence correction
  qt_solve(N, K, p, a0 / pr.dt + pr.nu * km2, R, R, tab(1, 0), tab(1, 1), tab(1, 2), tabG(1),
           w1, w2, w3, 0.0, 1.0);
  double2* V = X + NK;
  qt_solve(N, K, p, km2, R, V, tab(2, 0), tab(2, 1), tab(2, 2), tabG(2), w1, w2, w3, 0.0, -1.0);
  double2 s = czero();
  for (int n = p; n < N; n += 2) s = cfma((double)n * n, V[(size_t)n * K], s);
  const double* vh = g.vh + ((size_t)b * 4 + o) * NK + m;
  const double2 coef = cscl(s, -g.vhS[(((size_t)b * 4 + o) * 2 + p) * K + m]);
  for (int n = p; n < N; n += 2) {
    const size_t on = (size_t)n * K;
    V[on] = make_double2(fma(coef.x, vh[on], V[on].x), fma(coef.y, vh[on], V[on].y));
  }
}

// u = i (D v) / k from continuity (Eq. 3), m >= 1.  Advances the counter.
__global__ void k_uvel(GroupDev g) {
  const int b = blockIdx.y;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= g.K || g.status[b]) return;
  const int K = g.K, N = g.N;
  const size_t NK = (size_t)N * K;
  const MemberPrm pr = g.prm[b];
  double2* X = g.X + (size_t)b * 5 * NK + m;
  if (m == 0) {
    g.count[b] += 1;
    return;
  }
  const double ik = pr.lx / (2.0 * 3.14159265358979323846 * m);
  double2 p1 = czero(), p0 = czero();
  double2 av = X[NK + (size_t)(N - 1) * K];
  for (int n = N - 1; n >= 0; --n) {
    const size_t o = (size_t)n * K;
    const double2 d = (n == 0) ? cscl(p0, 0.5) : p0;
    X[o] = cscl(mul_i(d), ik);
    if (n >= 1) {
      const double2 nv = X[NK + o - K];
      const double2 pm = cfma(2.0 * n, av, p1);
      p1 = p0; p0 = pm; av = nv;
    }
  }
}

// ------------------------------------------------------------ diagnostics
// Partial reductions per member, one block each (deterministic order):
// part[0] = E by Clenshaw-Curtis in y (exact: 2N-1 points for degree 2N-2)
// and Parseval in x; part[1] = <Tr c>; part[2] = sum |state| (finiteness).
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

__global__ void __launch_bounds__(512) k_diag_part(GroupDev g) {
  const int b = blockIdx.x;
  if (g.status[b]) return;
  __shared__ double sh[32];
  const int K = g.K, N = g.N, Je = 2 * N - 1;
  const size_t NK = (size_t)N * K;
  const double2* DY = g.DY + (size_t)b * 4 * Je * K;
  double e = 0.0;
  for (int i = threadIdx.x; i < Je * K; i += blockDim.x) {
    const int j = i / K, m = i - j * K;
    const double2 uu = DY[(size_t)2 * Je * K + i], vv = DY[(size_t)3 * Je * K + i];
    const double w = (m == 0 ? 1.0 : 2.0) * g.ccw[j];
    e += w * (uu.x * uu.x + uu.y * uu.y + vv.x * vv.x + vv.y * vv.y);
  }
  e = block_sum(e, sh);
  const double2* X = g.X + (size_t)b * 5 * NK;
  double mt = 0.0;
  for (int n = threadIdx.x; n < N; n += blockDim.x) {
    if ((n & 1) == 0) mt += (X[2 * NK + (size_t)n * K].x + X[4 * NK + (size_t)n * K].x) * (2.0 / (1.0 - (double)n * n));
  }
  mt = block_sum(mt, sh);
  double cs = 0.0;
  for (size_t i = threadIdx.x; i < 5 * NK; i += blockDim.x) cs += fabs(X[i].x) + fabs(X[i].y);
  cs = block_sum(cs, sh);
  if (threadIdx.x == 0) {
    double* pp = g.part + (size_t)b * kPart;
    pp[0] = 0.25 * e;
    pp[1] = 0.5 * mt + 1.0;
    pp[2] = cs;
  }
}

// Per member: volume counts over the unpadded grid, mid-plane statistics,
// blow-up test, record.
__global__ void __launch_bounds__(512) k_diag_final(GroupDev g) {
  const int b = blockIdx.x;
  if (g.status[b]) return;
  __shared__ double sh[32];
  __shared__ double s_tau, s_stats[4];
  extern __shared__ double2 dsm[];
  const int K = g.K, N = g.N, nx = g.nx;
  const size_t NK = (size_t)N * K;
  const MemberPrm pr = g.prm[b];
  const double* cxx = g.DV + (size_t)b * 2 * N * nx;
  const double* cyy = cxx + (size_t)N * nx;
  const int npts = N * nx;
  // pass A: min, max, max|.|
  double mn = 1e308, mx = -1e308, ma = 0.0;
  bool nanf = false;
  for (int i = threadIdx.x; i < npts; i += blockDim.x) {
    const double t = cxx[i] + cyy[i] + 1.0;
    if (!(t == t)) nanf = true;
    mn = fmin(mn, t);
    mx = fmax(mx, t);
    ma = fmax(ma, fabs(t));
  }
  for (int o = 16; o > 0; o >>= 1) {
    mn = fmin(mn, __shfl_down_sync(0xffffffffu, mn, o));
    mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    ma = fmax(ma, __shfl_down_sync(0xffffffffu, ma, o));
  }
  nanf = __syncthreads_or(nanf);
  {
    __shared__ double smn[32], smx[32], sma[32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { smn[w] = mn; smx[w] = mx; sma[w] = ma; }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
        mn = fmin(mn, smn[i]); mx = fmax(mx, smx[i]); ma = fmax(ma, sma[i]);
      }
      s_stats[0] = nanf ? __longlong_as_double(0x7ff8000000000000LL) : mn;
      s_stats[1] = nanf ? __longlong_as_double(0x7ff8000000000000LL) : mx;
      s_tau = 1e-9 * ma;
    }
    __syncthreads();
  }
  const double tau = s_tau;
  // pass B: counts
  long long c3 = 0, c0 = 0, b3 = 0, b0 = 0;
  for (int i = threadIdx.x; i < npts; i += blockDim.x) {
    const double t = cxx[i] + cyy[i] + 1.0;
    c3 += (t < 3.0);
    c0 += (t < 0.0);
    b3 += (fabs(t - 3.0) <= tau);
    b0 += (fabs(t) <= tau);
  }
  double cnt4[4] = {(double)c3, (double)c0, (double)b3, (double)b0};
  double tot4[4];
  for (int q = 0; q < 4; ++q) tot4[q] = block_sum(cnt4[q], sh);
  // mid-plane spectra at y = 0: T_n(0) = cos(n pi/2), T_n'(0) = n sin(n pi/2)
  double2* L = dsm;              // 3 lines of nx
  double2* L2 = dsm + 3 * nx;    // ping-pong
  const double2* X = g.X + (size_t)b * 5 * NK;
  const double kfac = 2.0 * 3.14159265358979323846 / pr.lx;
  for (int i = threadIdx.x; i < 3 * nx; i += blockDim.x) L[i] = czero();
  __syncthreads();
  for (int m = threadIdx.x; m < K; m += blockDim.x) {
    double2 tr = czero(), u = czero(), v = czero(), uy = czero();
    for (int n = 0; n < N; ++n) {
      const size_t o = (size_t)n * K + m;
      const int r4 = n & 3;
      if (r4 == 0 || r4 == 2) {
        const double s = (r4 == 0) ? 1.0 : -1.0;
        tr = cfma(s, cadd(X[2 * NK + o], X[4 * NK + o]), tr);
        u = cfma(s, X[o], u);
        v = cfma(s, X[NK + o], v);
      } else {
        const double s = (r4 == 1) ? (double)n : -(double)n;
        uy = cfma(s, X[o], uy);
      }
    }
    const double km = kfac * m;
    double2 ux = cscl(mul_i(u), km), vx = cscl(mul_i(v), km);
    if (m == 0) { tr.x += 1.0; u = czero(); tr.y = v.y = uy.y = 0.0; ux = vx = czero(); }
    // lines: (Tr c, u') (v, ux) (vx, uy); Hermitian fill
    double2 F[6] = {tr, u, v, ux, vx, uy};
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
    const double* pp = g.part + (size_t)b * kPart;
    const long long step = g.count[b];
    ptt_diag r;
    r.step = step;
    r.t = step * pr.dt;
    r.energy = pp[0];
    r.mean_trc = pp[1];
    r.min_trc = s_stats[0];
    r.max_trc = s_stats[1];
    r.n_lt3 = (long long)tot4[0]; r.n_lt0 = (long long)tot4[1];
    r.n_band3 = (long long)tot4[2]; r.n_band0 = (long long)tot4[3];
    r.n_mid_lt3 = (long long)mct[0]; r.n_mid_lt0 = (long long)mct[1];
    r.n_mid_band3 = (long long)mct[2]; r.n_mid_band0 = (long long)mct[3];
    for (int qq = 0; qq < 8; ++qq)
      for (int k = 0; k < 4; ++k) r.mid_sums[qq][k] = (qq < 6) ? msum[qq][k] : 0.0;
    const bool fin = isfinite(pp[2]) && isfinite(pp[0]) && isfinite(r.max_trc);
    const bool blow = !fin || r.max_trc > pr.trc_max || sqrt(2.0 * pp[0]) > pr.u_max;
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

YJob make_yjob(const GroupDev& g, bool inverse, int M, int C, const FftPlan& pl) {
  YJob J{};
  J.K = g.K;
  J.N = g.N;
  J.M = M;
  J.inverse = inverse ? 1 : 0;
  J.C = C;
  J.pl = pl;
  J.status = g.status;
  return J;
}

}  // namespace

size_t smem_ycols(int C, int P) { return (size_t)(2 * C * P + 2 * C) * sizeof(double2); }
size_t smem_xfused(int Mx) { return (size_t)14 * Mx * sizeof(double2); }
size_t smem_xrows(int nl, int n) { return (size_t)2 * nl * n * sizeof(double2); }

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
  if ((e = optin(k_ycols, optin_bytes))) return e;
  if ((e = optin(k_xfused, optin_bytes))) return e;
  if ((e = optin(k_xrows, optin_bytes))) return e;
  if ((e = optin(k_diag_final, optin_bytes))) return e;
  return cudaSuccess;
}

// Stage s of one step for one group (see ptt.h: PTT_NSTAGES).
cudaError_t launch_stage(const GroupDev& g, int stage, cudaStream_t st, int* nl) {
  const int rows = g.M + 1;
  const size_t NK = (size_t)g.N * g.K;
  int n = 0;
  switch (stage) {
    case 0: {  // inverse y: 9 fields on the padded grid (two launches: 8 + 1)
      YJob J = make_yjob(g, true, g.M, g.Ccol, g.plP);
      J.src = g.X; J.dst = g.Yp;
      J.src_mstride = 5 * NK; J.dst_mstride = 9LL * rows * g.K;
      J.src_fstride = NK; J.dst_fstride = (long long)rows * g.K;
      const int sf[9] = {0, 1, 0, 2, 3, 4, 2, 3, 4};
      const int dv[9] = {0, 0, 1, 0, 0, 0, 1, 1, 1};
      for (int i = 0; i < 8; ++i) { J.src_field[i] = sf[i]; J.dst_field[i] = i; J.deriv[i] = dv[i]; }
      k_ycols<<<dim3(cdiv(g.K, g.Ccol), 8, g.nb), 256, smem_ycols(g.Ccol, g.P), st>>>(J);
      YJob J2 = J;
      J2.src_field[0] = sf[8]; J2.dst_field[0] = 8; J2.deriv[0] = dv[8];
      k_ycols<<<dim3(cdiv(g.K, g.Ccol), 1, g.nb), 256, smem_ycols(g.Ccol, g.P), st>>>(J2);
      n = 2;
      break;
    }
    case 1:
      k_xfused<<<dim3(rows, g.nb), 512, smem_xfused(g.Mx), st>>>(g);
      n = 1;
      break;
    case 2: {  // forward y of the 5 explicit fields
      YJob F = make_yjob(g, false, g.M, g.Ccol, g.plP);
      F.src = g.Zp; F.dst = g.NR;
      F.src_mstride = 5LL * rows * g.K; F.dst_mstride = 5 * NK;
      F.src_fstride = (long long)rows * g.K; F.dst_fstride = NK;
      for (int i = 0; i < 5; ++i) { F.src_field[i] = i; F.dst_field[i] = i; F.deriv[i] = 0; }
      k_ycols<<<dim3(cdiv(g.K, g.Ccol), 5, g.nb), 256, smem_ycols(g.Ccol, g.P), st>>>(F);
      n = 1;
      break;
    }
    case 3:
      k_rhs<<<dim3(cdiv(g.K, 128), g.nb), 128, 0, st>>>(g, 0);
      n = 1;
      break;
    case 4:
      k_solve<<<dim3(cdiv(g.K, 64), 8, g.nb), 64, 0, st>>>(g);
      n = 1;
      break;
    case 5:
      k_uvel<<<dim3(cdiv(g.K, 128), g.nb), 128, 0, st>>>(g);
      n = 1;
      break;
    case 6: {  // diagnostics
      const int Je = 2 * g.N - 1;
      YJob J = make_yjob(g, true, 2 * (g.N - 1), g.CcolE, g.plPe);
      J.src = g.X; J.dst = g.DY;
      J.src_mstride = 5 * NK; J.dst_mstride = 4LL * Je * g.K;
      J.src_fstride = NK; J.dst_fstride = (long long)Je * g.K;
      const int sf[4] = {2, 4, 0, 1};
      for (int i = 0; i < 4; ++i) { J.src_field[i] = sf[i]; J.dst_field[i] = i; J.deriv[i] = 0; }
      k_ycols<<<dim3(cdiv(g.K, g.CcolE), 4, g.nb), 256, smem_ycols(g.CcolE, g.Pe), st>>>(J);
      k_diag_part<<<g.nb, 512, 0, st>>>(g);
      XJob X{};
      X.srcC = g.DY; X.dstR = g.DV;
      X.src_mstride = 4LL * Je * g.K; X.dst_mstride = 2LL * g.N * g.nx;
      X.src_fstride = (long long)Je * g.K; X.dst_fstride = (long long)g.N * g.nx;
      X.src_rstep = 2; X.dst_rstep = 1;
      X.nf = 2; X.K = g.K; X.n = g.nx; X.c2r = 1; X.status = g.status; X.pl = g.plNx;
      k_xrows<<<dim3(g.N, g.nb), 256, smem_xrows(1, g.nx), st>>>(X);
      k_diag_final<<<g.nb, 512, smem_xrows(3, g.nx), st>>>(g);
      n = 4;
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
  k_rhs<<<dim3(cdiv(g.K, 128), g.nb), 128, 0, st>>>(g, 1);
  return cudaGetLastError();
}

cudaError_t launch_step(const GroupDev& g, cudaStream_t st, int* nl) {
  for (int s = 0; s < 6; ++s) {
    cudaError_t e = launch_stage(g, s, st, nl);
    if (e) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_diag(const GroupDev& g, cudaStream_t st, int* nl) {
  return launch_stage(g, 6, st, nl);
}

cudaError_t launch_reset_member(const GroupDev& g, int b, cudaStream_t st) {
  k_reset<<<1, 32, 0, st>>>(g, b);
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
  YJob J = make_yjob(g, false, g.N - 1, g.CcolE, g.plPu);
  J.status = nullptr;
  J.src = g.stageS; J.dst = g.X + (size_t)b * 5 * NK;
  J.src_fstride = NK; J.dst_fstride = NK;
  for (int i = 0; i < 5; ++i) { J.src_field[i] = i; J.dst_field[i] = i; J.deriv[i] = 0; }
  k_ycols<<<dim3(cdiv(g.K, g.CcolE), 5, 1), 256, smem_ycols(g.CcolE, g.Pu), st>>>(J);
  k_reset<<<1, 32, 0, st>>>(g, b);
  return cudaGetLastError();
}

cudaError_t launch_state_to_phys(const GroupDev& g, int b, cudaStream_t st) {
  const size_t NK = (size_t)g.N * g.K;
  YJob J = make_yjob(g, true, g.N - 1, g.CcolE, g.plPu);
  J.status = nullptr;
  J.src = g.X + (size_t)b * 5 * NK; J.dst = g.stageS;
  J.src_fstride = NK; J.dst_fstride = NK;
  for (int i = 0; i < 5; ++i) { J.src_field[i] = i; J.dst_field[i] = i; J.deriv[i] = 0; }
  k_ycols<<<dim3(cdiv(g.K, g.CcolE), 5, 1), 256, smem_ycols(g.CcolE, g.Pu), st>>>(J);
  XJob X{};
  X.srcC = g.stageS; X.dstR = g.stage;
  X.src_fstride = NK; X.dst_fstride = (long long)g.N * g.nx;
  X.src_rstep = 1; X.dst_rstep = 1;
  X.nf = 5; X.K = g.K; X.n = g.nx; X.c2r = 1; X.status = nullptr; X.pl = g.plNx;
  k_xrows<<<dim3(g.N, 1), 256, smem_xrows(3, g.nx), st>>>(X);
  return cudaGetLastError();
}

}  // namespace ptt
