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
#include <algorithm>
#include <cstdio>

#include "ptt_device.cuh"

namespace ptt {
namespace {

// ------------------------------------------------ fused x pass + products
// Yp fields: 0 u, 1 v, 2 du/dy, 3 cxx, 4 cxy, 5 cyy, 6 dcxx/dy, 7 dcxy/dy, 8 dcyy/dy.
// Physical lines (pairs re/im): (u, v) (uy, ux) (vx, cxx) (cxy, cyy)
// (cxx_y, cxy_y) (cyy_y, cxx_x) (cxy_x, cyy_x).
__constant__ int c_xsrc[14] = {0, 1, 2, 0, 1, 3, 4, 5, 6, 7, 8, 3, 4, 5};
__constant__ int c_xik[14] = {0, 0, 0, 1, 1, 0, 0, 0, 0, 0, 0, 1, 1, 1};

template <typename C2> __device__ __forceinline__ const C2* yp_ptr(const GroupDev& g);
template <> __device__ __forceinline__ const double2* yp_ptr<double2>(const GroupDev& g) { return g.Yp; }
template <> __device__ __forceinline__ const float2* yp_ptr<float2>(const GroupDev& g) { return g.Ypf; }
template <> __device__ __forceinline__ const dsc* yp_ptr<dsc>(const GroupDev& g) {
  return reinterpret_cast<const dsc*>(g.Yp);
}
template <typename C2> __device__ __forceinline__ C2* zp_ptr(const GroupDev& g);
template <> __device__ __forceinline__ double2* zp_ptr<double2>(const GroupDev& g) { return g.Zp; }
template <> __device__ __forceinline__ float2* zp_ptr<float2>(const GroupDev& g) { return g.Zpf; }
template <> __device__ __forceinline__ dsc* zp_ptr<dsc>(const GroupDev& g) { return reinterpret_cast<dsc*>(g.Zp); }

// The products of Eqs. 1-2 at one point of the padded grid, from the 14
// physical fields q = (u, v, du/dy, du/dx, dv/dx, c_xx, c_xy, c_yy, dc_xx/dy,
// dc_xy/dy, dc_yy/dy, dc_xx/dx, dc_xy/dx, dc_yy/dx) to (N_cxx, N_cxy, N_cyy,
// N_u, N_v): L_ij = du_i/dx_j (L_yy = -du/dx by continuity), relaxation
// factor 1 + eps Tr(c - I) with c_zz = 1.
template <typename T>
__device__ __forceinline__ void products2d(const T (&q)[14], T eps, T iwi, T (&o)[5]) {
  const T u = q[0], v = q[1], uy = q[2], ux = q[3], vx = q[4], cxx = q[5];
  const T cxy = q[6], cyy = q[7], cxx_y = q[8], cxy_y = q[9], cyy_y = q[10];
  const T cxx_x = q[11], cxy_x = q[12], cyy_x = q[13];
  const T rw = ((T)1 + eps * (cxx + cyy - (T)2)) * iwi;
  o[0] = -(u * cxx_x + v * cxx_y) + (T)2 * (ux * cxx + uy * cxy) - (cxx - (T)1) * rw;
  o[1] = -(u * cxy_x + v * cxy_y) + uy * cyy + vx * cxx - cxy * rw;
  o[2] = -(u * cyy_x + v * cyy_y) + (T)2 * (vx * cxy - ux * cyy) - (cyy - (T)1) * rw;
  // Eq. 2 advection
  o[3] = -(u * ux + v * uy);
  o[4] = -(u * vx - v * ux);
}

// C2 = double2: the FP64 path; C2 = float2: the mixed path (FP32 transforms
// and products, FP64 state and solves); C2 = dsc: the double-single path
// (FP64-accurate transforms and products on the FP32 pipe, PTT_FP64_DS).
// Mixed groups split the products into mean and fluctuation parts (mfl):
// the FP32 lines carry the fluctuations (their mean mode kk = 0 left out),
// the row's means come in FP64 from g.Ym, the mean products are formed once
// per row in FP64, and the mean column of the explicit terms goes to g.Zm
// in FP64 (the FP32 output's mean mode is left zero).
template <typename C2>
__device__ __forceinline__ void xfused_block(const GroupDev& g, Blk bk) {
  using T = typename RealOf<C2>::T;
  const int b = bk.y;
  if (g.status[b]) return;
  const int j = bk.x;
  const int K = g.K, Mx = g.Mx, rows = g.M;
  const MemberPrm pr = g.prm[b];
  extern __shared__ __align__(16) unsigned char smraw[];
  C2* A = reinterpret_cast<C2*>(smraw);
  C2* B = A + 7 * Mx;
  const C2* Y = yp_ptr<C2>(g) + (size_t)b * 9 * rows * K + (size_t)j * K;
  const T kfac = as_prec<T>(pr.kx1, pr.kx1f);
  const int tid = threadIdx.x, nt = blockDim.x;
  constexpr bool kSplit = std::is_same<C2, float2>::value;
  __shared__ float s_mq[14];    // the row's means as FP32 multipliers (split)
  __shared__ double s_nb[5];    // the row's mean products (split)
  if constexpr (kSplit) {
    const double2* ym = g.Ym + (size_t)b * 9 * rows + j;
    if (tid < 14) s_mq[tid] = c_xik[tid] ? 0.f : (float)ym[(size_t)c_xsrc[tid] * rows].x;
    if (tid == 32) {   // another warp: the mean products, in FP64
      double q[14], o[5];
      for (int i = 0; i < 14; ++i) q[i] = c_xik[i] ? 0.0 : ym[(size_t)c_xsrc[i] * rows].x;
      products2d<double>(q, pr.eps, pr.inv_wi, o);
      for (int i = 0; i < 5; ++i) s_nb[i] = o[i];
    }
  }
  // the padded middle K <= k <= Mx - K of every line is zero
  {
    const int nmid = Mx - 2 * K + 1;
    for (int i = tid; i < 7 * nmid; i += nt) {
      const int l = (int)fdiv((unsigned)i, fast_div((unsigned)nmid)), k = K + (i - l * nmid);
      A[l * Mx + k] = zero2<C2>();
    }
  }
  // items (line l, mode kk): the line's two fields loaded by one thread,
  // coalesced along kk, a batch of items in flight at once, then written
  // at k = kk and (conjugated) at Mx - kk
  {
    constexpr int kB = 4;   // items in flight per thread
    const int nitem = 7 * K;
    const FastDiv dK = fast_div((unsigned)K);
    for (int i0 = tid; i0 < nitem; i0 += kB * nt) {
      C2 F[kB], G[kB];
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const int it = i0 + u * nt;
        F[u] = G[u] = zero2<C2>();
        if (it < nitem) {
          const int l = (int)fdiv((unsigned)it, dK), kk = it - l * K;
          F[u] = Y[(size_t)c_xsrc[2 * l] * rows * K + kk];
          G[u] = Y[(size_t)c_xsrc[2 * l + 1] * rows * K + kk];
        }
      }
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const int it = i0 + u * nt;
        if (it >= nitem) continue;
        const int l = (int)fdiv((unsigned)it, dK), kk = it - l * K;
        C2 f = F[u], gg = G[u];
        if (kk == 0) { f.y = 0; gg.y = 0; }
        if (kSplit && kk == 0) { f.x = 0; gg.x = 0; }   // the mean is in g.Ym
        const T km = kfac * kk;
        if (c_xik[2 * l]) f = cscl(mul_i(f), km);
        if (c_xik[2 * l + 1]) gg = cscl(mul_i(gg), km);
        A[l * Mx + kk] = cadd(f, mul_i(gg));
        if (kk > 0) A[l * Mx + Mx - kk] = cadd(cconj(f), mul_i(cconj(gg)));
      }
    }
  }
  __syncthreads();
  // the padded modes K .. Mx - K are zero (plans of Mx start with radix 3
  // when Mx has no factor 5)
  C2* res = fft_lines<+1>(A, B, 7, Mx, g.plMx, g.plMx.radix[0] == 3);
  C2* oth = (res == A) ? B : A;
  const T eps = as_prec<T>(pr.eps, pr.epsf), iwi = as_prec<T>(pr.inv_wi, pr.inv_wif);
  for (int x = tid; x < Mx; x += nt) {
    T o[5];
    if constexpr (kSplit) {
      mfl q[14], om[5];
#pragma unroll
      for (int l = 0; l < 7; ++l) {
        const C2 h = res[l * Mx + x];
        q[2 * l] = mfl(s_mq[2 * l], h.x);
        q[2 * l + 1] = mfl(s_mq[2 * l + 1], h.y);
      }
      products2d<mfl>(q, mfl(pr.epsf, 0.f), mfl(pr.inv_wif, 0.f), om);
#pragma unroll
      for (int i = 0; i < 5; ++i) o[i] = om[i].f;
    } else {
      T q[14];
#pragma unroll
      for (int l = 0; l < 7; ++l) {
        const C2 h = res[l * Mx + x];
        q[2 * l] = h.x;
        q[2 * l + 1] = h.y;
      }
      products2d<T>(q, eps, iwi, o);
    }
    C2 o0, o1, o2;
    o0.x = o[0]; o0.y = o[1];
    o1.x = o[2]; o1.y = o[3];
    o2.x = o[4]; o2.y = 0;
    oth[x] = o0;
    oth[Mx + x] = o1;
    oth[2 * Mx + x] = o2;
  }
  __syncthreads();
  C2* r2 = fft_lines<-1>(oth, res, 3, Mx, g.plMx);
  C2* Z = zp_ptr<C2>(g) + (size_t)b * 5 * rows * K + (size_t)j * K;
  const T inv = as_prec<T>(g.invMx, g.invMxf);
  for (int i = tid; i < 3 * K; i += nt) {
    const int l = (int)fdiv((unsigned)i, fast_div((unsigned)K)), k = i - l * K;
    const C2 hk = r2[l * Mx + k];
    const C2 hm = cconj(r2[l * Mx + (k == 0 ? 0 : Mx - k)]);
    C2 F = cscl(cadd(hk, hm), (T)0.5 * inv);
    const C2 d = csub(hk, hm);
    C2 G;
    G.x = (T)0.5 * inv * d.y;
    G.y = (T)-0.5 * inv * d.x;
    if constexpr (kSplit) {
      if (k == 0) {   // mean column: the mean products plus the fluctuations' mean, FP64
        double2* zm = g.Zm + (size_t)b * 5 * rows + j;
        zm[(size_t)(2 * l) * rows] = make_double2(s_nb[2 * l] + (double)F.x, 0.0);
        if (l < 2) zm[(size_t)(2 * l + 1) * rows] = make_double2(s_nb[2 * l + 1] + (double)G.x, 0.0);
        F = zero2<C2>();
        G = zero2<C2>();
      }
    }
    Z[(size_t)(2 * l) * rows * K + k] = F;
    if (l < 2) Z[(size_t)(2 * l + 1) * rows * K + k] = G;
  }
}

template <typename C2>
__global__ void __launch_bounds__(512) k_xfused(GroupDev g) { xfused_block<C2>(g, this_blk()); }

template <typename C2>
__global__ void __launch_bounds__(512) k_xfused_multi(const GroupDev* __restrict__ gs, MultiMap mm) {
  Blk bk;
  const int q = multi_locate(mm, bk);
  xfused_block<C2>(gs[q], bk);
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
// CH: tau-scan rows per lane (register arrays of the solves; launch_spec
// picks the smallest of 2, 4, 8 that holds ny).  Two blocks per SM run the
// stage about 25 % faster than one block at the ~160 registers ptxas picks
// unbounded; CH = 2 and 4 take three (80 registers, a few spilled words,
// shared memory for three blocks up to ny = 257), CH = 8 two (its register
// arrays would spill heavily at 80).
template <int CH>
__device__ __forceinline__ void spec_block(const GroupDev& g, int mode, Blk bk) {
  const int b = bk.y;
  const int m = bk.x;
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
      const int w = (int)fdiv((unsigned)i, fast_div((unsigned)N)), n = i - w * N;
      tb[i] = qt[(size_t)w * NK + n];
    }
    const double* vh = g.vh + ((size_t)b * 4 + o) * NK + (size_t)m * N;
    for (int i = tid; i < N; i += nt) tb[9 * N + i] = vh[i];
  }
  __syncthreads();
  // derivatives, one warp per (column, parity): D c_xy -> sR[0], D c_yy -> sR[1],
  // D v -> sR[2], then D^2 v -> sq
  {
    const int warp = tid >> 5, par = warp & 1, col = warp >> 1;
    if (col == 0) warp_cheb_deriv_par(sc1, sR, N, par);
    else if (col == 1) warp_cheb_deriv_par(sc2, sR + N, N, par);
    else if (col == 2 && mode == 0 && m != 0) warp_cheb_deriv_par(sv, sR + 2 * N, N, par);
  }
  if (mode == 0 && m != 0) {
    __syncthreads();
    if (tid < 64) warp_cheb_deriv_par(sR + 2 * N, sq, N, tid >> 5);
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
  if (m != 0 && tid < 64) warp_cheb_deriv_par(shx, sR, N, tid >> 5);
  __syncthreads();
  for (int n = tid; n < N; n += nt)
    snq[n] = (m == 0) ? shx[n] : csub(cscl(mul_i(sR[n]), -km), cscl(shy[n], km2));
  __syncthreads();
  // history slot and SBDF sums
  if (g.f32 && m != 0) {   // mixed groups: the explicit-term history and its sum in FP32
    double2* E = g.Eh + ((size_t)slot * nb + b) * 4 * NK + (size_t)m * N;
    float2* Nf = reinterpret_cast<float2*>(g.Nh + ((size_t)slot * nb + b) * 4 * NK) + (size_t)m * N;
    const double idt = 1.0 / pr.dt;
    for (int i = tid; i < N; i += nt) {
      const double2 x[4] = {sc0[i], sc1[i], sc2[i], sq[i]};
      const double2 nn[4] = {NR[i], NR[NK + i], NR[2 * NK + i], snq[i]};
      double2 acc[4];
      float2 an[4];
      for (int s = 0; s < 4; ++s) {
        const float2 nf = f2_trunc(nn[s]);
        E[s * NK + i] = x[s];
        Nf[s * NK + i] = nf;
        acc[s] = cscl(x[s], -c_sa[o][1] * idt);
        an[s] = cscl(nf, c_sbf[o][0]);
      }
      for (int jj = 1; jj <= o; ++jj) {
        const size_t sl = (size_t)((slot - jj) & 3);
        const double2* Eo = g.Eh + (sl * nb + b) * 4 * NK + (size_t)m * N + i;
        const float2* No = reinterpret_cast<const float2*>(g.Nh + (sl * nb + b) * 4 * NK) + (size_t)m * N + i;
        const double ca = -c_sa[o][jj + 1] * idt;
        const float cb = c_sbf[o][jj];
        for (int s = 0; s < 4; ++s) {
          acc[s] = cfma(ca, Eo[s * NK], acc[s]);
          an[s] = cfma(cb, No[s * NK], an[s]);
        }
      }
      for (int s = 0; s < 4; ++s) sR[s * N + i] = cadd(acc[s], d2_exact(an[s]));
    }
  } else {
    // FP64 history; a mixed group's mean mode keeps it in FP64 in the second
    // half of the member's block (the FP32 view uses the first), stride N
    const size_t hs = g.f32 ? (size_t)N : NK;
    auto nd = [&](size_t sl) {
      double2* base = g.Nh + (sl * nb + b) * 4 * NK;
      return g.f32 ? base + 2 * NK : base + (size_t)m * N;
    };
    double2* E = g.Eh + ((size_t)slot * nb + b) * 4 * NK + (size_t)m * N;
    double2* Nn = nd((size_t)slot);
    const double idt = 1.0 / pr.dt;
    for (int i = tid; i < N; i += nt) {
      const double2 x[4] = {sc0[i], sc1[i], sc2[i], sq[i]};
      const double2 nn[4] = {NR[i], NR[NK + i], NR[2 * NK + i], snq[i]};
      double2 acc[4];
      for (int s = 0; s < 4; ++s) {
        E[s * NK + i] = x[s];
        Nn[s * hs + i] = nn[s];
        acc[s] = cfma(c_sb[o][0], nn[s], cscl(x[s], -c_sa[o][1] * idt));
      }
      for (int jj = 1; jj <= o; ++jj) {
        const size_t sl = (size_t)((slot - jj) & 3);
        const double2* Eo = g.Eh + (sl * nb + b) * 4 * NK + (size_t)m * N + i;
        const double2* No = nd(sl) + i;
        const double ca = -c_sa[o][jj + 1] * idt, cb = c_sb[o][jj];
        for (int s = 0; s < 4; ++s) acc[s] = cfma(cb, No[s * hs], cfma(ca, Eo[s * NK], acc[s]));
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
        warp_qt_solve<CH>(N, p, alpha, R, out, T0, T0 + N, T0 + 2 * N, G(0), w1, w2, w3, pr.dt / a0,
                      1.0);
      }
    } else if (m == 0) {
      warp_qt_solve<CH>(N, p, a0 / pr.dt, sR + 3 * N, shy, T1, T1 + N, T1 + 2 * N, G(1), w1, w2, w3,
                    0.0, 1.0);
      for (int n = p + 2 * lane; n < N; n += 64) sv[n] = czero();
    } else {
      double2* Rv = sR + 3 * N;
      warp_qt_solve<CH>(N, p, a0 / pr.dt + pr.nu * km2, Rv, Rv, T1, T1 + N, T1 + 2 * N, G(1), w1, w2,
                    w3, 0.0, 1.0);
      warp_qt_solve<CH>(N, p, km2, Rv, sv, T2, T2 + N, T2 + 2 * N, G(2), w1, w2, w3, 0.0, -1.0);
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
    if (tid < 64) warp_cheb_deriv_par(sv, sR, N, tid >> 5);
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

template <int CH>
__global__ void __launch_bounds__(256, (CH <= 4) ? 3 : 2) k_spec(GroupDev g, int mode) {
  spec_block<CH>(g, mode, this_blk());
}

template <int CH>
__global__ void __launch_bounds__(256, (CH <= 4) ? 3 : 2)
    k_spec_multi(const GroupDev* __restrict__ gs, MultiMap mm, int mode) {
  Blk bk;
  const int q = multi_locate(mm, bk);
  spec_block<CH>(gs[q], mode, bk);
}

// Advance the step counters (after every block of k_spec has read them).
__global__ void k_tick(GroupDev g) {
  const int b = threadIdx.x + blockIdx.x * blockDim.x;
  if (b < g.nb && !g.status[b]) g.count[b] += 1;
}

// The same for ng groups, one block per group.
__global__ void k_tick_multi(const GroupDev* __restrict__ gs, int ng) {
  const int q = blockIdx.x;
  if (q >= ng) return;
  const GroupDev& g = gs[q];
  for (int b = threadIdx.x; b < g.nb; b += blockDim.x)
    if (!g.status[b]) g.count[b] += 1;
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
// Diagnostics of one step, per member, as tiles (ntile blocks per member)
// with partial results in part[member][tile][kPart] reduced in a fixed
// order (deterministic):
//   DY: (u, v) on Me >= 2N-1 Gauss points (Fourier modes); DT, DV:
//       c_xx + c_yy on the unpadded Gauss-Lobatto rows (modes, then values).
//   E = <|u|^2/2> by Fejer's first rule in y (exact for degree 2N-2) and
//   Parseval in x; extrema of Tr c = c_xx + c_yy + 1; a non-finite test of
//   the state on the bit patterns; then the counts of Tr c < 3, < 0 and the
//   tie bands |Tr c - 3|, |Tr c| <= tau = 1e-9 max|Tr c|.
enum { P_E = 0, P_MIN, P_MAX, P_AMAX, P_BAD, P_C3, P_C0, P_B3, P_B0 };
constexpr int kMidLanes = 8, kMidModesPerBlock = 256 / kMidLanes;   // k_diag_mid, 256 threads
// Slot contents: P_E a double; P_MIN, P_MAX keys (dkey) of Tr c; P_AMAX the
// bits of max |Tr c|; P_BAD and the counts 64-bit integers.
__device__ __forceinline__ long long* islots(double* pp) { return reinterpret_cast<long long*>(pp); }
__device__ __forceinline__ const long long* islots(const double* pp) {
  return reinterpret_cast<const long long*>(pp);
}

__device__ __forceinline__ bool nonfinite(double x) {
  return (__double_as_longlong(x) & 0x7ff0000000000000LL) == 0x7ff0000000000000LL;
}

__device__ __forceinline__ void diag_part_block(const GroupDev& g, Blk bk) {
  const int b = bk.y, tile = bk.x;
  if (g.status[b]) return;
  const int K = g.K, N = g.N, nx = g.nx, Je = g.Me;
  const size_t NK = (size_t)N * K;
  const double2* DY = g.DY + (size_t)b * 2 * Je * K;
  double e = 0.0;
  KeyExt ext = keyext_empty();
  int bad = 0;
  // energy: DY fields 0 (u) and 1 (v) on the Me Gauss points (Fejer
  // weights); the modes m > 0 count twice (Parseval over +-m)
  {
    const unsigned tot = (unsigned)Je * K, per = (tot + g.ntile - 1) / g.ntile;
    const unsigned i0 = tile * per, i1 = min(tot, i0 + per);
    const FastDiv dK = fast_div((unsigned)K);
    double e0 = 0.0, e1 = 0.0;
    for (unsigned i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      const unsigned j = fdiv(i, dK), m = i - j * K;
      const double2 uu = DY[i], vv = DY[(size_t)Je * K + i];
      const double q = fma(uu.x, uu.x, fma(uu.y, uu.y, fma(vv.x, vv.x, vv.y * vv.y)));
      if (m == 0) e0 = fma(g.ccw[j], q, e0);
      else e1 = fma(g.ccw[j], q, e1);
    }
    e = fma(2.0, e1, e0);
  }
  // extrema of Tr c = (c_xx + c_yy) + 1 on the unpadded grid
  {
    const double* tr = g.DV + (size_t)b * N * nx;
    const long long tot = (long long)N * nx, per = (tot + g.ntile - 1) / g.ntile;
    const long long i0 = tile * per, i1 = min(tot, i0 + per);
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      const double t = tr[i] + 1.0;
      bad |= nonfinite(t);
      keyext_add(ext, t);
    }
  }
  // non-finite state values (integer test)
  {
    const double* X = reinterpret_cast<const double*>(g.X + (size_t)b * 5 * NK);
    const long long tot = 10LL * NK, per = (tot + g.ntile - 1) / g.ntile;
    const long long i0 = tile * per, i1 = min(tot, i0 + per);
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) bad |= nonfinite(X[i]);
  }
  __shared__ double sh[32];
  __shared__ long long shk[96];
  e = block_sum(e, sh);
  ext = block_keyext(ext, shk);
  bad = (int)block_isum(bad, shk);
  if (threadIdx.x == 0) {
    double* pp = g.part + ((size_t)b * g.ntile + tile) * kPart;
    pp[P_E] = e;
    islots(pp)[P_MIN] = ext.mn;
    islots(pp)[P_MAX] = ext.mx;
    islots(pp)[P_AMAX] = ext.ma;
    islots(pp)[P_BAD] = bad ? 1 : 0;
  }
}

__device__ __forceinline__ void diag_count_block(const GroupDev& g, Blk bk) {
  const int b = bk.y, tile = bk.x;
  if (g.status[b]) return;
  const int N = g.N, nx = g.nx;
  const TrBands B = tr_bands(1e-9 * block_tiles_amax(g.part + (size_t)b * g.ntile * kPart, g.ntile, P_AMAX));
  const double* tr = g.DV + (size_t)b * N * nx;
  const long long tot = (long long)N * nx, per = (tot + g.ntile - 1) / g.ntile;
  const long long i0 = tile * per, i1 = min(tot, i0 + per);
  TrCounts c{0, 0, 0, 0};
  for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) tr_count(c, tr[i] + 1.0, B);
  __shared__ long long shk[32];
  const long long c3 = block_isum(c.c3, shk), c0 = block_isum(c.c0, shk);
  const long long b3 = block_isum(c.b3, shk), b0 = block_isum(c.b0, shk);
  if (threadIdx.x == 0) {
    long long* pp = islots(g.part + ((size_t)b * g.ntile + tile) * kPart);
    pp[P_C3] = c3;
    pp[P_C0] = c0;
    pp[P_B3] = b3;
    pp[P_B0] = b0;
  }
}

// Mid-plane spectra at y = 0, kMidLanes lanes per (member, Fourier mode):
// T_n(0) = cos(n pi/2), T_n'(0) = n sin(n pi/2).  DM[b][q][m], q = Tr c, u, v,
// du/dy (Chebyshev sums; x derivatives and the mean are applied later).
// A mode's partial sums meet over its lanes only (three shuffle levels).
__device__ __forceinline__ double2 seg_sum2(double2 v) {
#pragma unroll
  for (int o = kMidLanes / 2; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o, kMidLanes);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o, kMidLanes);
  }
  return v;
}
__device__ __forceinline__ void diag_mid_block(const GroupDev& g, Blk bk) {
  const int b = bk.y;
  if (g.status[b]) return;
  const int sub = threadIdx.x & (kMidLanes - 1);
  const int m = bk.x * (blockDim.x / kMidLanes) + (threadIdx.x / kMidLanes);
  const int K = g.K, N = g.N;
  const bool on = m < K;   // every lane takes part in the shuffles
  const size_t NK = (size_t)N * K;
  const double2* X = g.X + (size_t)b * 5 * NK + (size_t)(on ? m : 0) * N;
  double2 tr = czero(), u = czero(), v = czero(), uy = czero();
  if (on) {
    // n = sub (mod kMidLanes): one residue of n mod 4 per lane
    const int r4 = sub & 3;
    if (r4 == 0 || r4 == 2) {
      const double s = (r4 == 0) ? 1.0 : -1.0;
      for (int n = sub; n < N; n += kMidLanes) {
        tr = cfma(s, cadd(X[2 * NK + n], X[4 * NK + n]), tr);
        u = cfma(s, X[n], u);
        v = cfma(s, X[NK + n], v);
      }
    } else {
      const double s = (r4 == 1) ? 1.0 : -1.0;
      for (int n = sub; n < N; n += kMidLanes) uy = cfma(s * n, X[n], uy);
    }
  }
  tr = seg_sum2(tr);
  u = seg_sum2(u);
  v = seg_sum2(v);
  uy = seg_sum2(uy);
  if (on && sub == 0) {
    double2* D = g.DM + (size_t)b * 4 * K + m;
    D[0] = tr;
    D[K] = u;
    D[2 * K] = v;
    D[3 * K] = uy;
  }
}

// Per member: reduce the tiles, <Tr c> from the mean mode, mid-plane
// statistics, blow-up test, record.
__device__ __forceinline__ void diag_final_block(const GroupDev& g, Blk bk) {
  const int b = bk.x;
  if (g.status[b]) return;
  __shared__ double sh[32];
  extern __shared__ double2 dsm[];
  const int K = g.K, N = g.N, nx = g.nx;
  const size_t NK = (size_t)N * K;
  const MemberPrm pr = g.prm[b];
  const double* pp = g.part + (size_t)b * g.ntile * kPart;
  // tile results, each thread a fixed set of tiles, then fixed-order trees
  // (the energy in FP64, extrema and counts on integers)
  __shared__ long long shk[96];
  double te = 0.0;
  KeyExt ext = keyext_empty();
  long long tbad = 0, tc[4] = {0, 0, 0, 0};
  for (int t = threadIdx.x; t < g.ntile; t += blockDim.x) {
    const double* q = pp + (size_t)t * kPart;
    const long long* qi = islots(q);
    te += q[P_E];
    keyext_merge(ext, KeyExt{qi[P_MIN], qi[P_MAX], qi[P_AMAX]});
    tbad |= qi[P_BAD];
    for (int k = 0; k < 4; ++k) tc[k] += qi[P_C3 + k];
  }
  te = block_sum(te, sh);
  ext = block_keyext(ext, shk);
  tbad = block_isum(tbad, shk);
  for (int k = 0; k < 4; ++k) tc[k] = block_isum(tc[k], shk);
  const TrBands B = tr_bands(1e-9 * __longlong_as_double(ext.ma));
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
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      L[l * nx + m] = cadd(F[2 * l], mul_i(F[2 * l + 1]));
      if (m > 0) L[l * nx + nx - m] = cadd(cconj(F[2 * l]), mul_i(cconj(F[2 * l + 1])));
    }
  }
  __syncthreads();
  double2* res = fft_lines<+1, double2, true>(L, L2, 3, nx, g.plNx);
  // mid-plane histograms of the 6 quantities (shared-memory counts)
  constexpr int HS = PTT_HIST_BINS + 2;
  __shared__ unsigned int hsm[6 * HS];
  __shared__ double hr[12];
  if (threadIdx.x < 12) hr[threadIdx.x] = g.hrange[(size_t)b * 16 + threadIdx.x];
  for (int i = threadIdx.x; i < 6 * HS; i += blockDim.x) hsm[i] = 0u;
  __syncthreads();
  bool hon = false;
#pragma unroll
  for (int q = 0; q < 6; ++q) hon |= (hr[2 * q] < hr[2 * q + 1]);
  // mid-plane counts (4, on integer keys) and power sums (6 quantities x 4
  // powers, padded to 32 for the reduce-scatter), one pass
  double acc[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) acc[k] = 0.0;
  TrCounts mc{0, 0, 0, 0};
  for (int x = threadIdx.x; x < nx; x += blockDim.x) {
    double q[6];
#pragma unroll
    for (int l = 0; l < 3; ++l) { q[2 * l] = res[l * nx + x].x; q[2 * l + 1] = res[l * nx + x].y; }
    if (hon) {
#pragma unroll
      for (int qq = 0; qq < 6; ++qq) {
        const int sl = hist_slot(q[qq], hr[2 * qq], hr[2 * qq + 1]);
        if (sl >= 0) atomicAdd(&hsm[qq * HS + sl], 1u);
      }
    }
    tr_count(mc, q[0], B);
#pragma unroll
    for (int qq = 0; qq < 6; ++qq) {
      const double a = q[qq], a2 = a * a;
      acc[4 * qq] += a;
      acc[4 * qq + 1] += a2;
      acc[4 * qq + 2] += a2 * a;
      acc[4 * qq + 3] += a2 * a2;
    }
  }
  __shared__ double red[8 * 32];
  block_sum_scatter(acc, red);   // its barriers also complete the shared counts
  const long long m3 = block_isum(mc.c3, shk), m0 = block_isum(mc.c0, shk);
  const long long mb3 = block_isum(mc.b3, shk), mb0 = block_isum(mc.b0, shk);
  if (hon) {
    unsigned long long* gh = g.hist + (size_t)b * 8 * HS;
    for (int i = threadIdx.x; i < 6 * HS; i += blockDim.x)
      if (hsm[i]) atomicAdd(&gh[i], (unsigned long long)hsm[i]);
  }
  if (threadIdx.x == 0) {
    const double e = 0.25 * te;
    const bool bad = (tbad != 0);
    const long long step = g.count[b];
    const double qnan = __longlong_as_double(0x7ff8000000000000LL);
    ptt_diag& r = g.ring[(size_t)b * kRing + (size_t)(step % kRing)];
    r.step = step;
    r.t = step * pr.dt;
    r.energy = e;
    r.mean_trc = 0.5 * mt + 1.0;
    r.min_trc = bad ? qnan : dkey_val(ext.mn);
    r.max_trc = bad ? qnan : dkey_val(ext.mx);
    r.n_lt3 = tc[0]; r.n_lt0 = tc[1];
    r.n_band3 = tc[2]; r.n_band0 = tc[3];
    r.n_mid_lt3 = m3; r.n_mid_lt0 = m0;
    r.n_mid_band3 = mb3; r.n_mid_band0 = mb0;
    for (int qq = 0; qq < 8; ++qq)
      for (int k = 0; k < 4; ++k) r.mid_sums[qq][k] = (qq < 6) ? red[4 * qq + k] : 0.0;
    const bool blow = bad || !isfinite(e) || r.max_trc > pr.trc_max || sqrt(2.0 * e) > pr.u_max;
    r.status = blow ? PTT_BLOWUP : PTT_OK;
    r.reserved = 0;
    if (blow) g.status[b] = 1;
    window_add(g.macc + (size_t)b * kMacc, r);
  }
}

__global__ void __launch_bounds__(256) k_diag_part(GroupDev g) { diag_part_block(g, this_blk()); }
__global__ void __launch_bounds__(256) k_diag_part_multi(const GroupDev* __restrict__ gs, MultiMap mm) {
  Blk bk;
  const int q = multi_locate(mm, bk);
  diag_part_block(gs[q], bk);
}
__global__ void __launch_bounds__(256) k_diag_count(GroupDev g) { diag_count_block(g, this_blk()); }
__global__ void __launch_bounds__(256) k_diag_count_multi(const GroupDev* __restrict__ gs, MultiMap mm) {
  Blk bk;
  const int q = multi_locate(mm, bk);
  diag_count_block(gs[q], bk);
}
__global__ void __launch_bounds__(256) k_diag_mid(GroupDev g) { diag_mid_block(g, this_blk()); }
__global__ void __launch_bounds__(256) k_diag_mid_multi(const GroupDev* __restrict__ gs, MultiMap mm) {
  Blk bk;
  const int q = multi_locate(mm, bk);
  diag_mid_block(gs[q], bk);
}
__global__ void __launch_bounds__(256) k_diag_final(GroupDev g) { diag_final_block(g, this_blk()); }
__global__ void __launch_bounds__(256) k_diag_final_multi(const GroupDev* __restrict__ gs, MultiMap mm) {
  Blk bk;
  const int q = multi_locate(mm, bk);
  diag_final_block(gs[q], bk);
}

// Spectral re-interpolation: destination coefficient (field, mode, n) from
// the source's same Fourier wavenumber(s) and Chebyshev index, zero where the
// source has none.  Modes: 2D m < K; 3D mx * nz + mz with mz in FFT order.
struct ResampleJob {
  const double2* src;   // source member's state [nf][KZs][Ns]
  double2* dst;         // destination member's state [nf][KZd][Nd]
  int nf;
  int Kd, nzd, Nd;      // destination x modes, z slots, Chebyshev modes
  int Ks, nzs, Ns;
};

__global__ void __launch_bounds__(256) k_resample(ResampleJob J) {
  const long long KZd = (long long)J.Kd * J.nzd, NKd = KZd * J.Nd;
  const long long NKs = (long long)J.Ks * J.nzs * J.Ns;
  const long long tot = (long long)J.nf * NKd;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
       i += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(i / NKd);
    const long long r = i - f * NKd;
    const int md = (int)(r / J.Nd), n = (int)(r - (long long)md * J.Nd);
    const int mx = md / J.nzd, mzd = md - mx * J.nzd;
    double2 v = czero();
    if (mx < J.Ks && n < J.Ns) {
      int mzs = -1;
      if (J.nzd == 1) {
        mzs = 0;
      } else if (mzd != J.nzd / 2) {
        const int sgn = (mzd < J.nzd / 2) ? mzd : mzd - J.nzd;   // signed wavenumber
        if (sgn > -J.nzs / 2 && sgn < J.nzs / 2) mzs = (sgn >= 0) ? sgn : sgn + J.nzs;
      }
      if (mzs >= 0) v = J.src[f * NKs + ((long long)mx * J.nzs + mzs) * J.Ns + n];
    }
    J.dst[i] = v;
  }
}

// Window statistics (Sec. 3: the moments of the mid-plane PDFs over a time
// window).  With n = npoints x records samples and raw moments
// m_p = S_p / n of the accumulated power sums S_p:
//   mean = m_1, var = m_2 - m_1^2, sd = sqrt(var),
//   skewness = (m_3 - 3 m_1 m_2 + 2 m_1^3) / sd^3,
//   kurtosis = (m_4 - 4 m_1 m_3 + 6 m_1^2 m_2 - 3 m_1^4) / var^2,
// (0 for both where var = 0), all in FP64; one thread per quantity.
__global__ void k_window_moments(const double* __restrict__ acc, double npoints,
                                 double* __restrict__ out) {
  const int q = threadIdx.x;
  const double nrec = acc[32];
  if (q < 8) {
    const double n = npoints * nrec;
    const double m1 = acc[4 * q] / n, m2 = acc[4 * q + 1] / n;
    const double m3 = acc[4 * q + 2] / n, m4 = acc[4 * q + 3] / n;
    const double var = fmax(m2 - m1 * m1, 0.0), sd = sqrt(var);
    const double c3 = m3 - 3.0 * m1 * m2 + 2.0 * m1 * m1 * m1;
    const double c4 = m4 - 4.0 * m1 * m3 + 6.0 * m1 * m1 * m2 - 3.0 * m1 * m1 * m1 * m1;
    out[4 * q] = m1;
    out[4 * q + 1] = sd;
    out[4 * q + 2] = sd > 0.0 ? c3 / (sd * sd * sd) : 0.0;
    out[4 * q + 3] = sd > 0.0 ? c4 / (var * var) : 0.0;
  }
  if (q == 0) out[32] = nrec;
}

// L1 distance between two histograms of each quantity, each normalised to
// unit total count: sum_i |a_i / A - b_i / B| over every slot (under- and
// overflow included); 0 if both are empty, 2 if only one is.  One warp per
// quantity, fixed-order shuffle trees.
__global__ void k_hist_l1(const unsigned long long* __restrict__ ha,
                          const unsigned long long* __restrict__ hb, double* __restrict__ out) {
  constexpr int HS = PTT_HIST_BINS + 2;
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned long long* a = ha + (size_t)q * HS;
  const unsigned long long* b = hb + (size_t)q * HS;
  double A = 0.0, B = 0.0;
  for (int i = lane; i < HS; i += 32) {
    A += (double)a[i];
    B += (double)b[i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    A += __shfl_xor_sync(0xffffffffu, A, o);
    B += __shfl_xor_sync(0xffffffffu, B, o);
  }
  double d = 0.0;
  if (A > 0.0 && B > 0.0)
    for (int i = lane; i < HS; i += 32) d += fabs((double)a[i] / A - (double)b[i] / B);
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  if (lane == 0) out[q] = (A > 0.0 && B > 0.0) ? d : ((A > 0.0) == (B > 0.0) ? 0.0 : 2.0);
}

__global__ void k_reset(GroupDev g, int b) {
  if (threadIdx.x == 0) {
    g.count[b] = 0;
    g.status[b] = 0;
  }
}


// Spectral coefficients (internal layout [member][field][m][n]) <-> values on
// a y grid stored [member][field][j][m].
YJob make_yjob(const GroupDev& g, bool inverse, int M, int C, const FftPlan& pl,
               const double2* tw4 = nullptr) {
  YJob J{};
  J.gauss = tw4 ? 1 : 0;
  J.tw4 = tw4;  // the quarter-period table of this direction
  J.tw4f = inverse ? g.tw4Pif : g.tw4Pf;
  J.tw4d = inverse ? g.tw4Pid : g.tw4Pd;
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
  for (int i = 0; i < kYFields; ++i) J.src_field2[i] = J.src_field3[i] = -1;
  return J;
}

}  // namespace

cudaError_t launch_resample(const GroupDev& d, int bd, const GroupDev& s, int bs, cudaStream_t st) {
  ResampleJob J;
  J.nf = (d.nz > 1) ? 9 : 5;
  J.Kd = d.K; J.nzd = d.nz; J.Nd = d.N;
  J.Ks = s.K; J.nzs = s.nz; J.Ns = s.N;
  J.src = s.X + (size_t)bs * J.nf * s.N * s.KZ;
  J.dst = d.X + (size_t)bd * J.nf * d.N * d.KZ;
  const long long tot = (long long)J.nf * d.KZ * d.N;
  const unsigned blocks = (unsigned)std::min<long long>((tot + 255) / 256, 152LL * 16);
  k_resample<<<blocks, 256, 0, st>>>(J);
  return cudaGetLastError();
}

cudaError_t launch_window_moments(const GroupDev& g, int b, double npoints, cudaStream_t st) {
  k_window_moments<<<1, 32, 0, st>>>(g.macc + (size_t)b * kMacc, npoints, g.statout);
  return cudaGetLastError();
}

cudaError_t launch_hist_l1(const unsigned long long* ha, const unsigned long long* hb, double* out,
                           cudaStream_t st) {
  k_hist_l1<<<1, 256, 0, st>>>(ha, hb, out);
  return cudaGetLastError();
}


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
  if ((e = optin(k_ycols<dsc>, optin_bytes))) return e;
  if ((e = optin(k_ycols<double2, true>, optin_bytes))) return e;
  if ((e = optin(k_ycols<dsc, true>, optin_bytes))) return e;
  if ((e = optin(k_ycols_multi<double2>, optin_bytes))) return e;
  if ((e = optin(k_ycols_multi<float2>, optin_bytes))) return e;
  if ((e = optin(k_ycols_multi<double2, true>, optin_bytes))) return e;
  if ((e = optin(k_xfused_multi<double2>, optin_bytes))) return e;
  if ((e = optin(k_xfused_multi<float2>, optin_bytes))) return e;
  if ((e = optin(k_xfused_multi<dsc>, optin_bytes))) return e;
  if ((e = optin(k_ycols_multi<dsc>, optin_bytes))) return e;
  if ((e = optin(k_ycols_multi<dsc, true>, optin_bytes))) return e;
  if ((e = optin(k_spec_multi<2>, optin_bytes))) return e;
  if ((e = optin(k_spec_multi<4>, optin_bytes))) return e;
  if ((e = optin(k_spec_multi<kMaxChunk>, optin_bytes))) return e;
  if ((e = optin(k_xrows_multi, optin_bytes))) return e;
  if ((e = optin(k_diag_final_multi, optin_bytes))) return e;
  if ((e = optin(k_xfused<double2>, optin_bytes))) return e;
  if ((e = optin(k_xfused<float2>, optin_bytes))) return e;
  if ((e = optin(k_xfused<dsc>, optin_bytes))) return e;
  if ((e = optin(k_xrows, optin_bytes))) return e;
  if ((e = optin(k_spec<2>, optin_bytes))) return e;
  if ((e = optin(k_spec<4>, optin_bytes))) return e;
  if ((e = optin(k_spec<kMaxChunk>, optin_bytes))) return e;
  if ((e = optin(k_diag_final, optin_bytes))) return e;
  return cudaSuccess;
}

// k_spec with the smallest tau-scan chunk that holds the group's rows:
// ceil((L - 1)/32) rows per lane with L = (ny + 1)/2 coefficients of parity 0.
// Tau-scan rows per lane of k_spec for a group's Chebyshev count.
static int spec_rows(const GroupDev& g) { return ((g.N + 1) / 2 - 1 + 31) / 32; }

static void launch_spec(const GroupDev& g, int mode, cudaStream_t st) {
  const int rows = spec_rows(g);
  const dim3 grid(g.K, g.nb);
  const size_t sm = smem_spec(g.N);
  if (rows <= 2) k_spec<2><<<grid, 256, sm, st>>>(g, mode);
  else if (rows <= 4) k_spec<4><<<grid, 256, sm, st>>>(g, mode);
  else k_spec<kMaxChunk><<<grid, 256, sm, st>>>(g, mode);
}

// Jobs of the y transforms and the Tr c x synthesis of a 2D group (shared by
// the per-group launches and the launches over all groups).
static YJob yjob_inverse(const GroupDev& g) {   // 9 fields on the padded Gauss grid
  const size_t NK = (size_t)g.N * g.K;
  YJob J = make_yjob(g, true, g.M, g.Ccol, g.plP, g.tw4Pi);
  J.src = g.X; J.dst = g.f32 ? (void*)g.Ypf : (void*)g.Yp;
  J.dst_f32 = g.ds ? kFmtDS : g.f32;
  J.src_mstride = 5 * NK; J.dst_mstride = 9LL * g.M * g.K;
  J.src_fstride = NK; J.dst_fstride = (long long)g.M * g.K;
  const int sf[9] = {0, 1, 0, 2, 3, 4, 2, 3, 4};
  const int dv[9] = {0, 0, 1, 0, 0, 0, 1, 1, 1};
  for (int i = 0; i < 9; ++i) { J.src_field[i] = sf[i]; J.dst_field[i] = i; J.deriv[i] = dv[i]; }
  return J;
}
static YJob yjob_forward(const GroupDev& g) {   // the 5 explicit fields to coefficients
  const size_t NK = (size_t)g.N * g.K;
  YJob F = make_yjob(g, false, g.M, g.Ccol, g.plP, g.tw4P);
  F.src = g.f32 ? (const void*)g.Zpf : (const void*)g.Zp; F.dst = g.NR;
  F.src_f32 = g.ds ? kFmtDS : g.f32;
  F.src_mstride = 5LL * g.M * g.K; F.dst_mstride = 5 * NK;
  F.src_fstride = (long long)g.M * g.K; F.dst_fstride = NK;
  for (int i = 0; i < 5; ++i) { F.src_field[i] = i; F.dst_field[i] = i; F.deriv[i] = 0; }
  return F;
}
// Mixed groups: the mean column (m = 0) of the inverse and forward y passes
// in double-single, FP64 in and out (g.Ym, g.Zm; see xfused_block).  One
// column per block; the narrow plan plPn (the double-single passes take
// radices up to 5).
static YJob yjob_mean_inverse(const GroupDev& g) {
  YJob J = yjob_inverse(g);
  J.K = 1; J.C = 1; J.pl = g.plPn;
  J.dst = g.Ym; J.dst_f32 = 0;
  J.dst_mstride = 9LL * g.M; J.dst_fstride = g.M;
  J.vm = 1; J.vj = 1;
  return J;
}
static YJob yjob_mean_forward(const GroupDev& g) {
  YJob F = yjob_forward(g);
  F.K = 1; F.C = 1; F.pl = g.plPn;
  F.src = g.Zm; F.src_f32 = 0;
  F.src_mstride = 5LL * g.M; F.src_fstride = g.M;
  F.vm = 1; F.vj = 1;
  return F;
}
static YJob yjob_energy(const GroupDev& g) {    // u, v on the Me Gauss points
  const size_t NK = (size_t)g.N * g.K;
  YJob J = make_yjob(g, true, g.Me, g.CcolE, g.plPe, g.tw4E);
  J.tw4f = g.tw4Ef;   // mixed groups transform in FP32 (the sums stay FP64)
  J.tw4d = g.tw4Ed;   // double-single groups in double-single
  J.src = g.X; J.dst = g.DY;
  J.src_mstride = 5 * NK; J.dst_mstride = 2LL * g.Me * g.K;
  J.src_fstride = NK; J.dst_fstride = (long long)g.Me * g.K;
  for (int i = 0; i < 2; ++i) { J.src_field[i] = i; J.dst_field[i] = i; J.deriv[i] = 0; }
  return J;
}
static YJob yjob_trc(const GroupDev& g) {       // c_xx + c_yy on the unpadded rows (DCT-I)
  const size_t NK = (size_t)g.N * g.K;
  YJob T = make_yjob(g, true, g.N - 1, g.CcolU, g.plPu);
  T.src = g.X; T.dst = g.DT;
  T.src_mstride = 5 * NK; T.dst_mstride = (long long)NK;
  T.src_fstride = NK; T.dst_fstride = 0;
  T.src_field[0] = 2; T.src_field2[0] = 4; T.dst_field[0] = 0; T.deriv[0] = 0;
  return T;
}
static XJob xjob_trc(const GroupDev& g) {       // Tr c rows to the unpadded x grid
  XJob X{};
  X.srcC = g.DT; X.dstR = g.DV;
  X.src_mstride = (long long)g.N * g.K; X.dst_mstride = (long long)g.N * g.nx;
  X.src_fstride = 0; X.dst_fstride = 0;
  X.src_rstep = 1; X.dst_rstep = 1;
  X.nf = 1; X.K = g.K; X.n = g.nx; X.c2r = 1; X.status = g.status; X.pl = g.plNx;
  X.pair_rows = 1; X.nrows = g.N;
  return X;
}


// Stage s of one step for one group (see ptt.h: PTT_NSTAGES).
cudaError_t launch_stage(const GroupDev& g, int stage, cudaStream_t st, int* nl) {
  const int rows = g.M;
  int n = 0;
  switch (stage) {
    case 0: {  // inverse y: 9 fields on the padded Gauss grid, one launch
      if (g.f32 && g.ymma) {
        cudaError_t e = launch_cheb_mma(g, true, st, g.nsm);
        if (e) return e;
        n = 1;
      } else {
        const YJob J = yjob_inverse(g);
        const size_t sm = smem_ycols(g.Ccol, g.M, g.f32);
        if (g.f32) k_ycols<float2><<<dim3(cdiv(g.K, g.Ccol), 9, g.nb), 256, sm, st>>>(J);
        else if (g.ds) k_ycols<dsc><<<dim3(cdiv(g.K, g.Ccol), 9, g.nb), 256, sm, st>>>(J);
        else k_ycols<double2><<<dim3(cdiv(g.K, g.Ccol), 9, g.nb), 256, sm, st>>>(J);
        n = 1;
      }
      if (g.f32) {   // the mean column in double-single
        k_ycols<dsc><<<dim3(1, 9, g.nb), 256, smem_ycols(1, g.M, 0), st>>>(yjob_mean_inverse(g));
        ++n;
      }
      break;
    }
    case 1:
      if (g.f32) k_xfused<float2><<<dim3(rows, g.nb), g.xthreads, smem_xfused(g.Mx, 1), st>>>(g);
      else if (g.ds) k_xfused<dsc><<<dim3(rows, g.nb), g.xthreads, smem_xfused(g.Mx, 0), st>>>(g);
      else k_xfused<double2><<<dim3(rows, g.nb), g.xthreads, smem_xfused(g.Mx, 0), st>>>(g);
      n = 1;
      break;
    case 2: {  // forward y of the 5 explicit fields
      if (g.f32 && g.ymma) {
        cudaError_t e = launch_cheb_mma(g, false, st, g.nsm);
        if (e) return e;
        n = 1;
      } else {
        const YJob F = yjob_forward(g);
        const size_t sm = smem_ycols(g.Ccol, g.M, g.f32);
        if (g.f32) k_ycols<float2><<<dim3(cdiv(g.K, g.Ccol), 5, g.nb), 256, sm, st>>>(F);
        else if (g.ds) k_ycols<dsc><<<dim3(cdiv(g.K, g.Ccol), 5, g.nb), 256, sm, st>>>(F);
        else k_ycols<double2><<<dim3(cdiv(g.K, g.Ccol), 5, g.nb), 256, sm, st>>>(F);
        n = 1;
      }
      if (g.f32) {   // the mean column in double-single, over the FP32 pass's zeros
        k_ycols<dsc><<<dim3(1, 5, g.nb), 256, smem_ycols(1, g.M, 0), st>>>(yjob_mean_forward(g));
        ++n;
      }
      break;
    }
    case 3:
      launch_spec(g, 0, st);
      k_tick<<<cdiv(g.nb, 128), 128, 0, st>>>(g);
      n = 2;
      break;
    case 4: {  // diagnostics, in order on one stream
      const DiagStreams d{{st, st, st}, {nullptr, nullptr, nullptr}};
      return launch_diag_split(g, d, nl);
    }
    default:
      return cudaErrorInvalidValue;
  }
  if (nl) *nl += n;
  return cudaGetLastError();
}

// Fork d.s[1], d.s[2] off d.s[0] (when distinct) before the parts, join after.
static cudaError_t diag_fork(const DiagStreams& d) {
  if (d.s[1] == d.s[0]) return cudaSuccess;
  cudaError_t e = cudaEventRecord(d.ev[0], d.s[0]);
  if (!e) e = cudaStreamWaitEvent(d.s[1], d.ev[0], 0);
  if (!e) e = cudaStreamWaitEvent(d.s[2], d.ev[0], 0);
  return e;
}
static cudaError_t diag_join(const DiagStreams& d) {
  if (d.s[1] == d.s[0]) return cudaSuccess;
  cudaError_t e = cudaEventRecord(d.ev[1], d.s[1]);
  if (!e) e = cudaEventRecord(d.ev[2], d.s[2]);
  if (!e) e = cudaStreamWaitEvent(d.s[0], d.ev[1], 0);
  if (!e) e = cudaStreamWaitEvent(d.s[0], d.ev[2], 0);
  return e;
}

// The diagnostics' y transforms (they write only DY, DT): u, v on the Me
// Gauss points of the energy quadrature; c_xx + c_yy on the unpadded
// Gauss-Lobatto rows (DCT-I).
static void diag_energy_y(const GroupDev& g, cudaStream_t st) {
  if (g.f32)
    k_ycols<float2><<<dim3(cdiv(g.K, g.CcolE), 2, g.nb), 256, smem_ycols(g.CcolE, g.Me, 1), st>>>(
        yjob_energy(g));
  else if (g.ds)
    k_ycols<dsc><<<dim3(cdiv(g.K, g.CcolE), 2, g.nb), 256, smem_ycols(g.CcolE, g.Me, 0), st>>>(
        yjob_energy(g));
  else
    k_ycols<double2><<<dim3(cdiv(g.K, g.CcolE), 2, g.nb), 256, smem_ycols(g.CcolE, g.Me, 0), st>>>(
        yjob_energy(g));
}
static void diag_trc_y(const GroupDev& g, cudaStream_t st) {
  if (g.ds || g.f32)   // double-single (FP64 in and out, FP64 sums downstream)
    k_ycols<dsc, true><<<dim3(cdiv(g.K, g.CcolU), 1, g.nb), 256, smem_ycols(g.CcolU, g.Pu, 0), st>>>(
        yjob_trc(g));
  else
    k_ycols<double2, true><<<dim3(cdiv(g.K, g.CcolU), 1, g.nb), 256, smem_ycols(g.CcolU, g.Pu, 0), st>>>(
        yjob_trc(g));
}

cudaError_t launch_diag_transforms(const GroupDev& g, cudaStream_t st) {
  diag_energy_y(g, st);
  diag_trc_y(g, st);
  return cudaGetLastError();
}

cudaError_t launch_diag_split(const GroupDev& g, const DiagStreams& d, int* nl) {
  cudaError_t e = diag_fork(d);
  if (e) return e;
  diag_energy_y(g, d.s[1]);
  // mid-plane sums per Fourier mode
  k_diag_mid<<<dim3(cdiv(g.K, kMidModesPerBlock), g.nb), 256, 0, d.s[2]>>>(g);
  // Tr c on the unpadded grid: y, then x
  diag_trc_y(g, d.s[0]);
  k_xrows<<<dim3(cdiv(g.N, 2), g.nb), 256, smem_xrows(1, g.nx), d.s[0]>>>(xjob_trc(g));
  if ((e = cudaGetLastError()) || (e = diag_join(d))) return e;
  k_diag_part<<<dim3(g.ntile, g.nb), 256, 0, d.s[0]>>>(g);
  k_diag_count<<<dim3(g.ntile, g.nb), 256, 0, d.s[0]>>>(g);
  k_diag_final<<<g.nb, 256, smem_xrows(3, g.nx), d.s[0]>>>(g);
  if (nl) *nl += 7;
  return cudaGetLastError();
}

// ------------------------------------------------- launches over all groups
struct Multi2DPlan {
  int ng = 0, f32 = 0, ds = 0;
  const GroupDev* dg = nullptr;
  // [6][ng]: inverse, forward, energy, Tr c, mean-column inverse and forward
  // (mixed groups)
  const YJob* dyj = nullptr;
  const XJob* dxj = nullptr;     // [ng]: Tr c x synthesis
  MultiMap inv, fwd, xf, spec[3], ye, yt, xr, mid, part, cnt, fin, ymi, ymf;
  size_t sm_inv = 0, sm_fwd = 0, sm_xf = 0, sm_spec[3] = {0, 0, 0}, sm_ye = 0, sm_yt = 0, sm_xr = 0,
         sm_fin = 0, sm_ym = 0;
};

int multi2d_max_groups() { return kMaxGroupsMulti; }

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t multi2d_bytes(int ng) {
  return align256((size_t)ng * sizeof(GroupDev)) + align256((size_t)6 * ng * sizeof(YJob)) +
         align256((size_t)ng * sizeof(XJob));
}

// Append group q with a launch grid (gx, gy, gz) to map mm.
static void mm_add(MultiMap& mm, int q, unsigned gx, unsigned gy, unsigned gz) {
  const int e = mm.ng++;
  mm.gid[e] = q;
  mm.gx[e] = (int)gx;
  mm.gy[e] = (int)gy;
  mm.gz[e] = (int)gz;
  mm.start[e + 1] = mm.start[e] + gx * gy * gz;
}

Multi2DPlan* multi2d_create(const std::vector<const GroupDev*>& groups, void* dev, cudaStream_t st,
                            cudaError_t* err) {
  *err = cudaSuccess;
  const int ng = (int)groups.size();
  if (ng < 1 || ng > kMaxGroupsMulti) { *err = cudaErrorInvalidValue; return nullptr; }
  Multi2DPlan* p = new Multi2DPlan();
  p->ng = ng;
  p->f32 = groups[0]->f32;
  p->ds = groups[0]->ds;
  std::vector<GroupDev> hg(ng);
  std::vector<YJob> hy(6 * (size_t)ng);
  std::vector<XJob> hx(ng);
  MultiMap* maps[] = {&p->inv, &p->fwd, &p->xf, &p->spec[0], &p->spec[1], &p->spec[2], &p->ye,
                      &p->yt, &p->xr, &p->mid, &p->part, &p->cnt, &p->fin, &p->ymi, &p->ymf};
  for (MultiMap* m : maps) { m->ng = 0; m->start[0] = 0; }
  // Each launch lists the groups with the costliest blocks first, so that
  // the blocks dispatched last, which set the launch's tail, are short ones.
  struct Ent { double cost; int q; unsigned gx, gy, gz; };
  std::vector<Ent> e_inv, e_fwd, e_xf, e_spec[3], e_ye, e_yt, e_xr, e_mid, e_part, e_fin, e_ymi, e_ymf;
  for (int q = 0; q < ng; ++q) {
    const GroupDev& g = *groups[q];
    if (g.nz != 1 || g.f32 != p->f32 || g.ds != p->ds || g.ymma) {
      delete p;
      *err = cudaErrorInvalidValue;
      return nullptr;
    }
    hg[q] = g;
    hy[q] = yjob_inverse(g);
    hy[ng + q] = yjob_forward(g);
    hy[2 * (size_t)ng + q] = yjob_energy(g);
    hy[3 * (size_t)ng + q] = yjob_trc(g);
    if (g.f32) {
      hy[4 * (size_t)ng + q] = yjob_mean_inverse(g);
      hy[5 * (size_t)ng + q] = yjob_mean_forward(g);
      e_ymi.push_back({(double)g.M, q, 1, 9, (unsigned)g.nb});
      e_ymf.push_back({(double)g.M, q, 1, 5, (unsigned)g.nb});
      p->sm_ym = std::max(p->sm_ym, smem_ycols(1, g.M, 0));
    }
    hx[q] = xjob_trc(g);
    e_inv.push_back({(double)g.Ccol * g.M, q, cdiv(g.K, g.Ccol), 9, (unsigned)g.nb});
    e_fwd.push_back({(double)g.Ccol * g.M, q, cdiv(g.K, g.Ccol), 5, (unsigned)g.nb});
    e_xf.push_back({(double)g.Mx, q, (unsigned)g.M, (unsigned)g.nb, 1});
    const int rows = spec_rows(g);
    const int cls = (rows <= 2) ? 0 : (rows <= 4) ? 1 : 2;
    e_spec[cls].push_back({(double)g.N, q, (unsigned)g.K, (unsigned)g.nb, 1});
    e_ye.push_back({(double)g.CcolE * g.Me, q, cdiv(g.K, g.CcolE), 2, (unsigned)g.nb});
    e_yt.push_back({(double)g.CcolU * g.Pu, q, cdiv(g.K, g.CcolU), 1, (unsigned)g.nb});
    e_xr.push_back({(double)g.nx, q, cdiv(g.N, 2), (unsigned)g.nb, 1});
    e_mid.push_back({(double)g.N, q, cdiv(g.K, kMidModesPerBlock), (unsigned)g.nb, 1});
    e_part.push_back({(double)g.N * g.nx / g.ntile, q, (unsigned)g.ntile, (unsigned)g.nb, 1});
    e_fin.push_back({(double)g.nx + g.ntile, q, (unsigned)g.nb, 1, 1});
    p->sm_inv = std::max(p->sm_inv, smem_ycols(g.Ccol, g.M, g.f32));
    p->sm_fwd = p->sm_inv;
    p->sm_xf = std::max(p->sm_xf, smem_xfused(g.Mx, g.f32));
    p->sm_spec[cls] = std::max(p->sm_spec[cls], smem_spec(g.N));
    p->sm_ye = std::max(p->sm_ye, smem_ycols(g.CcolE, g.Me, g.f32));
    p->sm_yt = std::max(p->sm_yt, smem_ycols(g.CcolU, g.Pu, 0));
    p->sm_xr = std::max(p->sm_xr, smem_xrows(1, g.nx));
    p->sm_fin = std::max(p->sm_fin, smem_xrows(3, g.nx));
  }
  auto fill = [](MultiMap& m, std::vector<Ent>& v) {
    std::stable_sort(v.begin(), v.end(), [](const Ent& a, const Ent& b) { return a.cost > b.cost; });
    for (const Ent& x : v) mm_add(m, x.q, x.gx, x.gy, x.gz);
  };
  fill(p->inv, e_inv);
  fill(p->fwd, e_fwd);
  fill(p->xf, e_xf);
  for (int c = 0; c < 3; ++c) fill(p->spec[c], e_spec[c]);
  fill(p->ye, e_ye);
  fill(p->yt, e_yt);
  fill(p->xr, e_xr);
  fill(p->mid, e_mid);
  fill(p->part, e_part);
  std::vector<Ent> e_cnt = e_part;
  fill(p->cnt, e_cnt);
  fill(p->fin, e_fin);
  fill(p->ymi, e_ymi);
  fill(p->ymf, e_ymf);
  char* b = static_cast<char*>(dev);
  p->dg = reinterpret_cast<const GroupDev*>(b);
  p->dyj = reinterpret_cast<const YJob*>(b + align256((size_t)ng * sizeof(GroupDev)));
  p->dxj = reinterpret_cast<const XJob*>(b + align256((size_t)ng * sizeof(GroupDev)) +
                                          align256((size_t)6 * ng * sizeof(YJob)));
  cudaError_t e = cudaMemcpyAsync((void*)p->dg, hg.data(), hg.size() * sizeof(GroupDev),
                                  cudaMemcpyHostToDevice, st);
  if (!e) e = cudaMemcpyAsync((void*)p->dyj, hy.data(), hy.size() * sizeof(YJob), cudaMemcpyHostToDevice, st);
  if (!e) e = cudaMemcpyAsync((void*)p->dxj, hx.data(), hx.size() * sizeof(XJob), cudaMemcpyHostToDevice, st);
  if (!e) e = cudaStreamSynchronize(st);   // the host vectors go out of scope
  if (e) { delete p; *err = e; return nullptr; }
  return p;
}

void multi2d_destroy(Multi2DPlan* p) { delete p; }

static unsigned mm_blocks(const MultiMap& m) { return m.start[m.ng]; }

cudaError_t launch_stage_multi(const Multi2DPlan* p, int stage, cudaStream_t st, int* nl) {
  int n = 0;
  const int ng = p->ng;
  switch (stage) {
    case 0:
      if (p->f32) k_ycols_multi<float2><<<mm_blocks(p->inv), 256, p->sm_inv, st>>>(p->dyj, p->inv);
      else if (p->ds) k_ycols_multi<dsc><<<mm_blocks(p->inv), 256, p->sm_inv, st>>>(p->dyj, p->inv);
      else k_ycols_multi<double2><<<mm_blocks(p->inv), 256, p->sm_inv, st>>>(p->dyj, p->inv);
      n = 1;
      if (p->ymi.ng) {   // mixed groups: the mean columns in double-single
        k_ycols_multi<dsc><<<mm_blocks(p->ymi), 256, p->sm_ym, st>>>(p->dyj + 4 * ng, p->ymi);
        ++n;
      }
      break;
    case 1:
      if (p->f32) k_xfused_multi<float2><<<mm_blocks(p->xf), 512, p->sm_xf, st>>>(p->dg, p->xf);
      else if (p->ds) k_xfused_multi<dsc><<<mm_blocks(p->xf), 512, p->sm_xf, st>>>(p->dg, p->xf);
      else k_xfused_multi<double2><<<mm_blocks(p->xf), 512, p->sm_xf, st>>>(p->dg, p->xf);
      n = 1;
      break;
    case 2:
      if (p->f32) k_ycols_multi<float2><<<mm_blocks(p->fwd), 256, p->sm_fwd, st>>>(p->dyj + ng, p->fwd);
      else if (p->ds) k_ycols_multi<dsc><<<mm_blocks(p->fwd), 256, p->sm_fwd, st>>>(p->dyj + ng, p->fwd);
      else k_ycols_multi<double2><<<mm_blocks(p->fwd), 256, p->sm_fwd, st>>>(p->dyj + ng, p->fwd);
      n = 1;
      if (p->ymf.ng) {
        k_ycols_multi<dsc><<<mm_blocks(p->ymf), 256, p->sm_ym, st>>>(p->dyj + 5 * ng, p->ymf);
        ++n;
      }
      break;
    case 3:
      if (p->spec[0].ng) { k_spec_multi<2><<<mm_blocks(p->spec[0]), 256, p->sm_spec[0], st>>>(p->dg, p->spec[0], 0); ++n; }
      if (p->spec[1].ng) { k_spec_multi<4><<<mm_blocks(p->spec[1]), 256, p->sm_spec[1], st>>>(p->dg, p->spec[1], 0); ++n; }
      if (p->spec[2].ng) {
        k_spec_multi<kMaxChunk><<<mm_blocks(p->spec[2]), 256, p->sm_spec[2], st>>>(p->dg, p->spec[2], 0);
        ++n;
      }
      k_tick_multi<<<ng, 128, 0, st>>>(p->dg, ng);
      ++n;
      break;
    case 4: {
      const DiagStreams d{{st, st, st}, {nullptr, nullptr, nullptr}};
      return launch_diag_multi(p, d, nl);
    }
    default:
      return cudaErrorInvalidValue;
  }
  if (nl) *nl += n;
  return cudaGetLastError();
}

cudaError_t launch_diag_multi(const Multi2DPlan* p, const DiagStreams& d, int* nl) {
  const int ng = p->ng;
  cudaError_t e = diag_fork(d);
  if (e) return e;
  if (p->f32) k_ycols_multi<float2><<<mm_blocks(p->ye), 256, p->sm_ye, d.s[1]>>>(p->dyj + 2 * ng, p->ye);
  else if (p->ds) k_ycols_multi<dsc><<<mm_blocks(p->ye), 256, p->sm_ye, d.s[1]>>>(p->dyj + 2 * ng, p->ye);
  else k_ycols_multi<double2><<<mm_blocks(p->ye), 256, p->sm_ye, d.s[1]>>>(p->dyj + 2 * ng, p->ye);
  k_diag_mid_multi<<<mm_blocks(p->mid), 256, 0, d.s[2]>>>(p->dg, p->mid);
  if (p->ds || p->f32)
    k_ycols_multi<dsc, true><<<mm_blocks(p->yt), 256, p->sm_yt, d.s[0]>>>(p->dyj + 3 * ng, p->yt);
  else k_ycols_multi<double2, true><<<mm_blocks(p->yt), 256, p->sm_yt, d.s[0]>>>(p->dyj + 3 * ng, p->yt);
  k_xrows_multi<<<mm_blocks(p->xr), 256, p->sm_xr, d.s[0]>>>(p->dxj, p->xr);
  if ((e = cudaGetLastError()) || (e = diag_join(d))) return e;
  k_diag_part_multi<<<mm_blocks(p->part), 256, 0, d.s[0]>>>(p->dg, p->part);
  k_diag_count_multi<<<mm_blocks(p->cnt), 256, 0, d.s[0]>>>(p->dg, p->cnt);
  k_diag_final_multi<<<mm_blocks(p->fin), 256, p->sm_fin, d.s[0]>>>(p->dg, p->fin);
  if (nl) *nl += 7;
  return cudaGetLastError();
}

cudaError_t launch_explicit(const GroupDev& g, cudaStream_t st) {
  for (int s = 0; s < 3; ++s) {
    cudaError_t e = launch_stage(g, s, st, nullptr);
    if (e) return e;
  }
  launch_spec(g, 1, st);
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
  k_ycols<double2, true><<<dim3(cdiv(g.K, g.CcolU), 5, 1), 256, smem_ycols(g.CcolU, g.Pu, 0), st>>>(J);
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
  k_ycols<double2, true><<<dim3(cdiv(g.K, g.CcolU), 5, 1), 256, smem_ycols(g.CcolU, g.Pu, 0), st>>>(J);
  XJob X{};
  X.srcC = g.stageS; X.dstR = g.stage;
  X.src_fstride = NK; X.dst_fstride = (long long)g.N * g.nx;
  X.src_rstep = 1; X.dst_rstep = 1;
  X.nf = 5; X.K = g.K; X.n = g.nx; X.c2r = 1; X.status = nullptr; X.pl = g.plNx;
  k_xrows<<<dim3(g.N, 1), 256, smem_xrows(3, g.nx), st>>>(X);
  return cudaGetLastError();
}

}  // namespace ptt
