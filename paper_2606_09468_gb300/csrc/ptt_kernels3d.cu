// Device code of the 3D pseudo-spectral sPTT channel step (sm_103a).
//
// Nine fields u, v, w, c_xx, c_xy, c_xz, c_yy, c_yz, c_zz; spectral arrays
// [member][field][mode][n] with mode = mx * nz + mz (mx < nx/2, mz in FFT
// order, the Nyquist slot nz/2 kept zero).  One step (Sec. 2):
//   k_ycols  (inverse)  17 columns per mode on the padded Gauss y grid
//                       (9 fields and 8 y-derivatives; d/dy of v follows from
//                       continuity)
//   k_zcols  (inverse)  per (y row, mx) line: 26 z syntheses of length Mz
//                       (the 17 fields and 9 z-derivatives)
//   k_xfused3           per (y, z) row: 35 physical fields (9 more
//                       x-derivatives), the products of Eqs. 1-2, 9 forward
//                       x transforms
//   k_zcols  (forward), k_ycols (forward): back to truncated spectral terms
//   k_spec3             per mode: explicit linear terms, SBDF sums, tau solves
//                       (six c, phi-v with the influence correction, eta; U and
//                       W on the mean mode), u and w from continuity and eta
//   k_tick              step counters
// followed by the Sec. 3 diagnostics over the nx x ny x nz grid and the
// (x, z) mid-plane.
#include <cstdio>

#include "ptt_device.cuh"

namespace ptt {
namespace {

// ------------------------------------------------------------ z lines
// Inverse: src [field][j][mx*nz + mz] (modes) -> dst [field][j][z][mx] (values
// at Mz points, optional d/dz).  Forward: src [field][j][z][mx] (values) ->
// dst [field][j][mx*nz + mz] (modes, truncated, Nyquist slot zero).
struct ZJob {
  const void* src;
  void* dst;
  int src_f32, dst_f32;
  long long src_mstride, dst_mstride;  // per member (elements)
  long long src_fstride, dst_fstride;  // per field (elements)
  int src_field[32];
  int dst_field[32];
  int dz[32];         // inverse: transform d/dz of the field
  int K, nz, Mz;      // x modes, z modes, z points
  double inv;         // forward: 1 / Mz (host-computed), and its FP32 rounding
  float invf;
  int inverse;
  int C;              // mx lines per block
  int rows;           // y rows per field
  const int* status;
  const MemberPrm* prm;
  FftPlan pl;         // length Mz
  // mixed groups' step passes (mean/fluctuation split, see k_xfused3):
  // mean = 1, inverse: the kx = 0 line leaves its kz = 0 (mean) mode out;
  // mean = 2, forward: the kx = 0 line's mean mode is added in FP64 to
  // zm[member][dst field][row] and left zero in dst
  int mean;
  double2* zm;
};

// BIG: unpadded z length nz (radices 7, 11, 13 possible); the padded length
// Mz of the step runs without it.
template <typename CT, bool BIG = false>
__global__ void __launch_bounds__(256) k_zcols(ZJob J) {
  using T = typename RealOf<CT>::T;
  const int b = blockIdx.z;
  if (J.status && J.status[b]) return;
  const int f = blockIdx.y / J.rows;
  const int j = blockIdx.y - f * J.rows;
  const int C = J.C, K = J.K, nz = J.nz, Mz = J.Mz;
  const int m0 = blockIdx.x * C;
  const int nc = min(C, K - m0);
  extern __shared__ __align__(16) unsigned char smraw[];
  CT* A = reinterpret_cast<CT*>(smraw);
  CT* B = A + (size_t)C * Mz;
  const size_t es = (J.src_f32 == 1) ? sizeof(float2) : sizeof(double2);
  const size_t ed = (J.dst_f32 == 1) ? sizeof(float2) : sizeof(double2);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int hz = nz / 2;
  if (J.inverse) {
    const void* src = static_cast<const char*>(J.src) +
        (b * J.src_mstride + J.src_field[f] * J.src_fstride + (long long)j * K * nz) * es;
    void* dst = static_cast<char*>(J.dst) +
        (b * J.dst_mstride + J.dst_field[f] * J.dst_fstride + (long long)j * Mz * K) * ed;
    const T kfac = as_prec<T>(J.prm[b].kz1, J.prm[b].kz1f);
    const int dz = J.dz[f];
    for (int i = tid; i < C * Mz; i += nt) A[i] = zero2<CT>();
    __syncthreads();
    const bool skip0 = (J.mean == 1 && m0 == 0);
    for (int i = tid; i < C * nz; i += nt) {
      const int c = (int)fdiv((unsigned)i, fast_div((unsigned)nz)), mz = i - c * nz;
      if (c < nc && mz != hz && !(skip0 && c == 0 && mz == 0)) {
        const int s = (mz < hz) ? mz : mz - nz;
        CT v = ld2<CT>(src, (long long)(m0 + c) * nz + mz, J.src_f32);
        if (dz) v = cscl(mul_i(v), kfac * (T)s);
        A[c * Mz + (s >= 0 ? s : s + Mz)] = v;
      }
    }
    __syncthreads();
    // padded synthesis (Mz >= 3 nz/2): the slots nz/2 .. Mz - nz/2 are zero
    CT* res = fft_lines<+1, CT, BIG>(A, B, C, Mz, J.pl, J.pl.radix[0] == 3 && Mz >= 3 * hz);
    for (int i = tid; i < Mz * C; i += nt) {
      const int z = (int)fdiv((unsigned)i, fast_div((unsigned)C)), c = i - z * C;
      if (c < nc) st2<CT>(dst, (long long)z * K + m0 + c, J.dst_f32, res[c * Mz + z]);
    }
  } else {
    const void* src = static_cast<const char*>(J.src) +
        (b * J.src_mstride + J.src_field[f] * J.src_fstride + (long long)j * Mz * K) * es;
    void* dst = static_cast<char*>(J.dst) +
        (b * J.dst_mstride + J.dst_field[f] * J.dst_fstride + (long long)j * K * nz) * ed;
    for (int i = tid; i < Mz * C; i += nt) {
      const int z = (int)fdiv((unsigned)i, fast_div((unsigned)C)), c = i - z * C;
      A[c * Mz + z] = (c < nc) ? ld2<CT>(src, (long long)z * K + m0 + c, J.src_f32) : zero2<CT>();
    }
    __syncthreads();
    CT* res = fft_lines<-1, CT, BIG>(A, B, C, Mz, J.pl);
    const T inv = as_prec<T>(J.inv, J.invf);
    for (int i = tid; i < C * nz; i += nt) {
      const int c = (int)fdiv((unsigned)i, fast_div((unsigned)nz)), mz = i - c * nz;
      if (c < nc) {
        CT v = zero2<CT>();
        if (mz != hz) {
          const int s = (mz < hz) ? mz : mz - nz;
          v = cscl(res[c * Mz + (s >= 0 ? s : s + Mz)], inv);
        }
        if constexpr (std::is_same<CT, float2>::value) {
          if (J.mean == 2 && m0 + c == 0 && mz == 0) {
            J.zm[((size_t)b * 9 + J.dst_field[f]) * J.rows + j].x += (double)v.x;
            v = zero2<CT>();
          }
        }
        st2<CT>(dst, (long long)(m0 + c) * nz + mz, J.dst_f32, v);
      }
    }
  }
}

// ------------------------------------------------ fused x pass + products
// Z3 fields (26): 0 u, 1 v, 2 w, 3 cxx, 4 cxy, 5 cxz, 6 cyy, 7 cyz, 8 czz,
// 9 uy, 10 wy, 11-16 c_y (xx, xy, xz, yy, yz, zz), 17 uz, 18 vz, 19 wz,
// 20-25 c_z.  Physical fields (35): the 26 plus x-derivatives of fields 0-8
// (26 ux, 27 vx, 28 wx, 29-34 c_x), packed in pairs into 18 complex lines.
// W3 outputs (9): N_cxx, N_cxy, N_cxz, N_cyy, N_cyz, N_czz, N_u, N_v, N_w.
template <typename C2> __device__ __forceinline__ const C2* z3_ptr(const GroupDev& g);
template <> __device__ __forceinline__ const double2* z3_ptr<double2>(const GroupDev& g) { return g.Z3; }
template <> __device__ __forceinline__ const float2* z3_ptr<float2>(const GroupDev& g) { return g.Z3f; }
template <> __device__ __forceinline__ const dsc* z3_ptr<dsc>(const GroupDev& g) {
  return reinterpret_cast<const dsc*>(g.Z3);
}
template <typename C2> __device__ __forceinline__ C2* w3_ptr(const GroupDev& g);
template <> __device__ __forceinline__ double2* w3_ptr<double2>(const GroupDev& g) { return g.W3; }
template <> __device__ __forceinline__ float2* w3_ptr<float2>(const GroupDev& g) { return g.W3f; }
template <> __device__ __forceinline__ dsc* w3_ptr<dsc>(const GroupDev& g) { return reinterpret_cast<dsc*>(g.W3); }

// The products of Eqs. 1-2 at one point from the 35 physical fields q (Z3
// order, then the x-derivatives of fields 0-8 at 26-34; q[35] unused) to
// N_cxx, N_cxy, N_cxz, N_cyy, N_cyz, N_czz, N_u, N_v, N_w.
template <typename T>
__device__ __forceinline__ void products3d(const T (&q)[36], T eps, T iwi, T (&out)[9]) {
  const T u = q[0], v = q[1], w = q[2];
  const T C[3][3] = {{q[3], q[4], q[5]}, {q[4], q[6], q[7]}, {q[5], q[7], q[8]}};
  const T ux = q[26], vx = q[27], wx = q[28];
  const T uy = q[9], wy = q[10];
  const T uz = q[17], vz = q[18], wz = q[19];
  // L_ij = d u_i / d x_j, L_yy = -ux - wz (Eq. 3)
  const T L[3][3] = {{ux, uy, uz}, {vx, -ux - wz, vz}, {wx, wy, wz}};
  const T rw = ((T)1 + eps * (q[3] + q[6] + q[8] - (T)3)) * iwi;
  // components in storage order xx, xy, xz, yy, yz, zz; gradients in q
  const int ci[6] = {0, 0, 0, 1, 1, 2}, cj2[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const int i = ci[c], jj = cj2[c];
    const T adv = u * q[29 + c] + v * q[11 + c] + w * q[20 + c];
    T st = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) st += L[i][k] * C[k][jj] + C[i][k] * L[jj][k];
    const T dlt = (i == jj) ? (T)1 : (T)0;
    out[c] = -adv + st - (C[i][jj] - dlt) * rw;
  }
  // Eq. 2 advection: -(u . grad) u_i = -sum_k u_k L_ik
  const T uu[3] = {u, v, w};
#pragma unroll
  for (int i = 0; i < 3; ++i) out[6 + i] = -(uu[0] * L[i][0] + uu[1] * L[i][1] + uu[2] * L[i][2]);
}

// IP: the lines stay in one buffer and every FFT pass works in place
// (fft_lines_inplace; kIpThreads threads), for the FP64 lines too long for
// two buffers in shared memory (Mx up to kIpMaxN).
template <typename C2, bool IP = false>
__global__ void __launch_bounds__(512) k_xfused3(GroupDev g) {
  using T = typename RealOf<C2>::T;
  const int b = blockIdx.y;
  if (g.status[b]) return;
  const int row = blockIdx.x;  // j * Mz + z
  const int K = g.K, Mx = g.Mx;
  const long long plane = (long long)g.M * g.Mz * K;  // one field of one member
  const MemberPrm pr = g.prm[b];
  extern __shared__ __align__(16) unsigned char smraw[];
  C2* A = reinterpret_cast<C2*>(smraw);
  C2* B = A + 18 * Mx;
  const C2* Z = z3_ptr<C2>(g) + (size_t)b * 26 * plane + (size_t)row * K;
  const T kfac = as_prec<T>(pr.kx1, pr.kx1f);
  const int tid = threadIdx.x, nt = blockDim.x;
  // mixed groups: mean/fluctuation split of the products (see xfused_block
  // in the 2D kernels): the z pass left the mean mode out of the lines, the
  // means of the 17 y-pass fields at this row's y come from g.Ym (the z- and
  // x-derivatives have zero mean), the mean products go to g.Zm (written by
  // the rows at z = 0; the forward z pass adds the fluctuations' mean)
  constexpr bool kSplit = std::is_same<C2, float2>::value;
  __shared__ float s_mq[17];
  if constexpr (kSplit) {
    const int jy = row / g.Mz;
    const double2* ym = g.Ym + (size_t)b * 17 * g.M + jy;
    if (tid < 17) s_mq[tid] = (float)ym[(size_t)tid * g.M].x;
    if (tid == 32 && row - jy * g.Mz == 0) {
      double q[36], o[9];
      for (int i = 0; i < 36; ++i) q[i] = (i < 17) ? ym[(size_t)i * g.M].x : 0.0;
      products3d<double>(q, pr.eps, pr.inv_wi, o);
      double2* zm = g.Zm + (size_t)b * 9 * g.M + jy;
      for (int i = 0; i < 9; ++i) zm[(size_t)i * g.M] = make_double2(o[i], 0.0);
    }
  }
  // the padded middle K <= k <= Mx - K of every line is zero
  {
    const int nmid = Mx - 2 * K + 1;
    for (int i = tid; i < 18 * nmid; i += nt) {
      const int l = (int)fdiv((unsigned)i, fast_div((unsigned)nmid)), k = K + (i - l * nmid);
      A[l * Mx + k] = zero2<C2>();
    }
  }
  // lines 0-12: the 26 loaded fields in pairs (2l, 2l+1); line 13 + r
  // (r < 5): their x-derivatives i k (fields 2r, 2r+1; line 17 field 8
  // alone).  Items (l < 13, mode kk): both fields' coefficients loaded by
  // one thread, coalesced along kk, a batch of items in flight at once, then
  // written at k = kk and (conjugated) at Mx - kk.
  {
    constexpr int kB = 4;   // items in flight per thread
    const int nitem = 13 * K;
    const FastDiv dK = fast_div((unsigned)K);
    for (int i0 = tid; i0 < nitem; i0 += kB * nt) {
      C2 F[kB], G[kB];
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const int it = i0 + u * nt;
        F[u] = G[u] = zero2<C2>();
        if (it < nitem) {
          const int l = (int)fdiv((unsigned)it, dK), kk = it - l * K;
          F[u] = Z[(size_t)(2 * l) * plane + kk];
          G[u] = Z[(size_t)(2 * l + 1) * plane + kk];
        }
      }
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const int it = i0 + u * nt;
        if (it >= nitem) continue;
        const int l = (int)fdiv((unsigned)it, dK), kk = it - l * K;
        C2 f = F[u], gg = G[u];
        if (kk == 0) { f.y = 0; gg.y = 0; }
        A[l * Mx + kk] = cadd(f, mul_i(gg));
        if (kk > 0) A[l * Mx + Mx - kk] = cadd(cconj(f), mul_i(cconj(gg)));
        if (l < 5) {
          const T fk = kfac * (T)kk;
          C2 df = cscl(mul_i(F[u]), fk), dg = cscl(mul_i(G[u]), fk);
          if (l == 4) dg = zero2<C2>();
          if (kk == 0) { df.y = 0; dg.y = 0; }
          const int ld = 13 + l;
          A[ld * Mx + kk] = cadd(df, mul_i(dg));
          if (kk > 0) A[ld * Mx + Mx - kk] = cadd(cconj(df), mul_i(cconj(dg)));
        }
      }
    }
  }
  __syncthreads();
  C2* res;
  C2* oth;
  if constexpr (IP) {
    fft_lines_inplace<+1>(A, 18, Mx, g.plMx, g.plMx.radix[0] == 3);
    res = oth = A;   // each column x is read and rewritten by one thread
  } else {
    res = fft_lines<+1>(A, B, 18, Mx, g.plMx, g.plMx.radix[0] == 3);
    oth = (res == A) ? B : A;
  }
  const T eps = as_prec<T>(pr.eps, pr.epsf), iwi = as_prec<T>(pr.inv_wi, pr.inv_wif);
  for (int x = tid; x < Mx; x += nt) {
    T out[9];
    if constexpr (kSplit) {
      mfl q[36], om[9];
#pragma unroll
      for (int l = 0; l < 18; ++l) {
        const C2 h = res[l * Mx + x];
        q[2 * l] = mfl(2 * l < 17 ? s_mq[2 * l] : 0.f, h.x);
        q[2 * l + 1] = mfl(2 * l + 1 < 17 ? s_mq[2 * l + 1] : 0.f, h.y);
      }
      products3d<mfl>(q, mfl(pr.epsf, 0.f), mfl(pr.inv_wif, 0.f), om);
#pragma unroll
      for (int i = 0; i < 9; ++i) out[i] = om[i].f;
    } else {
      T q[36];
#pragma unroll
      for (int l = 0; l < 18; ++l) {
        const C2 h = res[l * Mx + x];
        q[2 * l] = h.x;
        q[2 * l + 1] = h.y;
      }
      products3d<T>(q, eps, iwi, out);
    }
#pragma unroll
    for (int l = 0; l < 5; ++l) {
      C2 o;
      o.x = out[2 * l];
      o.y = (2 * l + 1 < 9) ? out[2 * l + 1] : (T)0;
      oth[l * Mx + x] = o;
    }
  }
  __syncthreads();
  C2* r2;
  if constexpr (IP) {
    fft_lines_inplace<-1>(oth, 5, Mx, g.plMx);
    r2 = oth;
  } else {
    r2 = fft_lines<-1>(oth, res, 5, Mx, g.plMx);
  }
  C2* W = w3_ptr<C2>(g) + (size_t)b * 9 * plane + (size_t)row * K;
  const T inv = as_prec<T>(g.invMx, g.invMxf);
  for (int i = tid; i < 5 * K; i += nt) {
    const int l = (int)fdiv((unsigned)i, fast_div((unsigned)K)), k = i - l * K;
    const C2 hk = r2[l * Mx + k];
    const C2 hm = cconj(r2[l * Mx + (k == 0 ? 0 : Mx - k)]);
    const C2 F = cscl(cadd(hk, hm), (T)0.5 * inv);
    const C2 d = csub(hk, hm);
    C2 G;
    G.x = (T)0.5 * inv * d.y;
    G.y = (T)-0.5 * inv * d.x;
    W[(size_t)(2 * l) * plane + k] = F;
    if (2 * l + 1 < 9) W[(size_t)(2 * l + 1) * plane + k] = G;
  }
}

// ---------------------------------------------- per-mode spectral stage
// Explicit terms (Eq. 2): H_i = N_u,i + gam (div c)_i (+ 2/Re on the mean
// mode, x); forcings of the evolved velocity quantities (k != 0):
// q1 = -D(i kx H_x + i kz H_z) - k^2 H_y (phi = (D^2 - k^2) v),
// q2 = i kz H_x - i kx H_z (eta = i kz u - i kx w); mean mode: H_x, H_z.
// Evolved (8): c (6), q1 state, q2 state.  Solves per mode: six c (wall rows
// of Eq. 1 at kappa = 0), phi -> v -> influence correction (k != 0) or U,
// eta (k != 0) or W; then u = i (kx Dv - kz eta)/k^2, w = i (kz Dv + kx eta)/k^2.
//
// A block takes 16 modes; lane l of every warp owns mode l/2 of the block and
// Chebyshev parity l%2, and each warp runs one component task of a phase, so
// all recurrences run lane-sequentially with full warps.  Per-mode scratch
// columns live in SS (workspace; L2-resident while the block runs):
enum {
  S3_DCXY = 0, S3_DCYY, S3_DCYZ, S3_DV, S3_D2V,   // derivatives of the state
  S3_HX, S3_HY, S3_HZ,                             // explicit momentum terms H
  S3_Q1, S3_Q2,                                    // evolved q1, q2 (state)
  S3_F1T, S3_F1, S3_F2,                            // forcings of q1, q2
  S3_R,                                            // 8 SBDF sums (13..20)
  S3_DVN = S3_R + 8,                               // D of the new v
  S3_PHI, S3_ETA,                                  // solved phi, eta
  kScr3                                            // 24 columns per mode
};
constexpr int kModesPerBlock = 16;

__global__ void __launch_bounds__(256) k_spec3(GroupDev g, int mode) {
  const int b = blockIdx.y;
  if (g.status[b]) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = lane & 1;
  const int KZ = g.KZ, N = g.N, nb = g.nb, nz = g.nz;
  const size_t NK = (size_t)N * KZ;
  const int md0 = blockIdx.x * kModesPerBlock + (lane >> 1);
  const bool inb = md0 < KZ;
  const int md = inb ? md0 : KZ - 1;
  const int mx = md / nz, mzi = md - mx * nz, hz = nz / 2;
  const bool nyq = (mzi == hz);
  const bool act = inb && !nyq;
  const bool mean = (mx == 0 && mzi == 0);
  const MemberPrm pr = g.prm[b];
  const long long cnt = g.count[b];
  const int slot = (int)(cnt & 3);
  const int o = (cnt < 3) ? (int)cnt : 3;
  const int sz = (mzi < hz) ? mzi : mzi - nz;
  const double kx = 2.0 * 3.14159265358979323846 * mx / pr.lx;
  const double kz = 2.0 * 3.14159265358979323846 * sz / pr.lz;
  const double k2 = kx * kx + kz * kz;
  const size_t col = (size_t)md * N;
  double2* X = g.X + (size_t)b * 9 * NK + col;          // field f at X + f * NK
  const double2* NR = g.NR + (size_t)b * 9 * NK + col;
  double2* S = g.SS + (size_t)b * kScr3 * NK + col;     // scratch column a at S + a * NK
  auto SC = [&](int a) { return S + (size_t)a * NK; };
  const double gam = pr.gam;

  // the dropped Nyquist slot stays zero
  if (warp == 0 && inb && nyq) {
    if (mode == 0) {
      for (int f = 0; f < 9; ++f)
        for (int n = p; n < N; n += 2) X[f * NK + n] = czero();
      double2* E = g.Eh + ((size_t)slot * nb + b) * 8 * NK + col;
      double2* Nn = g.Nh + ((size_t)slot * nb + b) * 8 * NK + col;
      for (int s2 = 0; s2 < 8; ++s2)
        for (int n = p; n < N; n += 2) { E[s2 * NK + n] = czero(); Nn[s2 * NK + n] = czero(); }
    } else {
      double2* R = g.Rb + (size_t)b * 4 * NK + col;
      for (int f = 0; f < 3; ++f)
        for (int n = p; n < N; n += 2) R[f * NK + n] = czero();
    }
  }
  // phase 1: derivatives D c_xy, D c_yy, D c_yz; D v, D^2 v
  if (act) {
    if (warp == 0) lane_cheb_deriv(X + 4 * NK, SC(S3_DCXY), N, p);
    else if (warp == 1) lane_cheb_deriv(X + 6 * NK, SC(S3_DCYY), N, p);
    else if (warp == 2) lane_cheb_deriv(X + 7 * NK, SC(S3_DCYZ), N, p);
  }
  if (warp == 3) {
    const bool d = act && mode == 0 && !mean;
    if (d) lane_cheb_deriv(X + NK, SC(S3_DV), N, p);
    __syncwarp();
    if (d) lane_cheb_deriv(SC(S3_DV), SC(S3_D2V), N, p);
  }
  __syncthreads();
  // Element-wise phases split the lane's column over the eight warps: warp w
  // takes elements [w c8, (w + 1) c8) of its lane's parity (n = p + 2 i), so
  // every warp keeps loads in flight (one warp per column waited on each
  // element in turn).
  const int Lp = (N - p + 1) / 2;
  const int c8 = (Lp + 7) / 8;
  const int e0 = min(Lp, warp * c8), e1 = min(Lp, e0 + c8);
  // phase 2: H (all three components), evolved q1, q2
  if (act) {
    const double2* __restrict__ Xc = X;
    const double2* __restrict__ Sd = S;
    double2* __restrict__ Sw = S;
    const double fx = mean ? pr.forcing : 0.0;
    for (int i = e0; i < e1; ++i) {
      const int n = p + 2 * i;
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        // (div c)_i = i kx c_xi + D c_yi + i kz c_zi
        const int cx = (t == 0) ? 3 : (t == 1) ? 4 : 5;     // c_xx, c_xy, c_xz
        const int cz = (t == 0) ? 5 : (t == 1) ? 7 : 8;     // c_xz, c_yz, c_zz
        const double2 dv = cadd(cscl(mul_i(Xc[(size_t)cx * NK + n]), kx),
                                cadd(Sd[(size_t)(S3_DCXY + t) * NK + n],
                                     cscl(mul_i(Xc[(size_t)cz * NK + n]), kz)));
        double2 h = cfma(gam, dv, NR[(size_t)(6 + t) * NK + n]);
        if (t == 0 && n == 0) h.x += fx;
        Sw[(size_t)(S3_HX + t) * NK + n] = h;
      }
      if (mode == 0) {
        Sw[(size_t)S3_Q1 * NK + n] = mean ? Xc[n] : cfma(-k2, Xc[NK + n], Sd[(size_t)S3_D2V * NK + n]);
        Sw[(size_t)S3_Q2 * NK + n] =
            mean ? Xc[2 * NK + n] : csub(cscl(mul_i(Xc[n]), kz), cscl(mul_i(Xc[2 * NK + n]), kx));
      }
    }
  }
  __syncthreads();
  if (mode == 1) {   // explicit right-hand side only: H -> Rb
    if (act && warp < 3) {
      double2* R = g.Rb + (size_t)b * 4 * NK + col + (size_t)warp * NK;
      const double2* H = SC(S3_HX + warp);
      for (int n = p; n < N; n += 2) R[n] = H[n];
    }
    return;
  }
  // phase 3: forcings of q1 = -D(i kx H_x + i kz H_z) - k^2 H_y and of
  // q2 = i kz H_x - i kx H_z (mean mode: H_x, H_z): the element-wise parts
  // over all warps, the derivative on warp 0
  {
    const double2* __restrict__ Hx = SC(S3_HX);
    const double2* __restrict__ Hy = SC(S3_HY);
    const double2* __restrict__ Hz = SC(S3_HZ);
    double2* __restrict__ t = SC(S3_F1T);
    double2* __restrict__ f2 = SC(S3_F2);
    if (act)
      for (int i = e0; i < e1; ++i) {
        const int n = p + 2 * i;
        if (!mean) t[n] = cadd(cscl(mul_i(Hx[n]), kx), cscl(mul_i(Hz[n]), kz));
        f2[n] = mean ? Hz[n] : csub(cscl(mul_i(Hx[n]), kz), cscl(mul_i(Hz[n]), kx));
      }
    __syncthreads();
    if (warp == 0 && act && !mean) lane_cheb_deriv(SC(S3_F1T), SC(S3_F1), N, p);
    __syncthreads();
    double2* __restrict__ f = SC(S3_F1);
    if (act)
      for (int i = e0; i < e1; ++i) {
        const int n = p + 2 * i;
        f[n] = mean ? Hx[n] : csub(cscl(f[n], -1.0), cscl(Hy[n], k2));
      }
  }
  __syncthreads();
  // phase 4: history slot and SBDF sums, warp s for evolved quantity s
  if (act) {
    const int s2 = warp;
    const double2* x = (s2 < 6) ? X + (size_t)(3 + s2) * NK : SC(S3_Q1 + (s2 - 6));
    const double2* nn = (s2 < 6) ? NR + (size_t)s2 * NK : SC(S3_F1 + (s2 - 6));
    double2* E = g.Eh + ((size_t)slot * nb + b) * 8 * NK + (size_t)s2 * NK + col;
    double2* R = SC(S3_R + s2);
    const double2* Eo[3];
    for (int jj = 1; jj <= 3; ++jj) {
      const size_t sl = (size_t)((slot - jj) & 3);
      Eo[jj - 1] = g.Eh + (sl * nb + b) * 8 * NK + (size_t)s2 * NK + col;
    }
    // FP64 history in every form: in a mixed group the mean mode would need
    // it in FP64 (its explicit terms carry the 2/Re forcing and the
    // 10^4-sized stretching), and its lanes share warps with the other
    // modes, so an FP32 history elsewhere would diverge the warps of the
    // block holding the mean mode, which sets the launch's time (one wave
    // at 128 x 97 x 64: measured 0.60 -> 0.66 ms)
    double2* Nn = g.Nh + ((size_t)slot * nb + b) * 8 * NK + (size_t)s2 * NK + col;
    const double2* No[3];
    for (int jj = 1; jj <= 3; ++jj) {
      const size_t sl = (size_t)((slot - jj) & 3);
      No[jj - 1] = g.Nh + (sl * nb + b) * 8 * NK + (size_t)s2 * NK + col;
    }
    lane_sbdf_any(o, N, p, 1.0 / pr.dt, x, nn, E, Nn, Eo, No, R);
  }
  __syncthreads();
  // phase 5: tau solves; warps 0-5 the c components, 6 q1, 7 q2
  if (act) {
    const double* w1 = g.wrow;
    const double* w2 = g.wrow + N;
    const double* w3 = g.wrow + 2 * N;
    const double a0 = c_sa[o][0];
    const double* qt = g.qt + ((size_t)b * 4 + o) * 3 * 3 * NK + col;
    auto T = [&](int sys, int k) { return qt + (size_t)(sys * 3 + k) * NK; };
    auto G = [&](int sys) { return g.qtG[((((size_t)b * 4 + o) * 3 + sys) * 2 + p) * KZ + md]; };
    if (warp < 6) {
      const double2* R = SC(S3_R + warp);
      double2* out = X + (size_t)(3 + warp) * NK;
      const double alpha = a0 / pr.dt + pr.kappa * k2;
      if (pr.kappa == 0.0) {
        const double ia = 1.0 / alpha;
        for (int n = p; n < N; n += 2) out[n] = cscl(R[n], ia);
      } else {
        lane_qt_solve(N, p, alpha, R, out, T(0, 0), T(0, 1), T(0, 2), G(0), w1, w2, w3,
                      pr.dt / a0, 1.0);
      }
    } else if (warp == 6) {
      double2* R1 = SC(S3_R + 6);
      if (mean) {
        lane_qt_solve(N, p, a0 / pr.dt, R1, X, T(1, 0), T(1, 1), T(1, 2), G(1), w1, w2, w3, 0.0, 1.0);
        for (int n = p; n < N; n += 2) X[NK + n] = czero();
      } else {
        double2* v = X + NK;
        double2* phi = SC(S3_PHI);
        lane_qt_solve(N, p, a0 / pr.dt + pr.nu * k2, R1, phi, T(1, 0), T(1, 1), T(1, 2), G(1), w1,
                      w2, w3, 0.0, 1.0);
        lane_qt_solve(N, p, k2, phi, v, T(2, 0), T(2, 1), T(2, 2), G(2), w1, w2, w3, 0.0, -1.0);
        double2 sacc = czero();
        for (int n = p; n < N; n += 2) sacc = cfma((double)n * n, v[n], sacc);
        const double* vh = g.vh + ((size_t)b * 4 + o) * NK + col;
        const double2 coef = cscl(sacc, -g.vhS[(((size_t)b * 4 + o) * 2 + p) * KZ + md]);
        for (int n = p; n < N; n += 2)
          v[n] = make_double2(fma(coef.x, vh[n], v[n].x), fma(coef.y, vh[n], v[n].y));
      }
    } else {
      double2* R2 = SC(S3_R + 7);
      const double alpha = mean ? a0 / pr.dt : a0 / pr.dt + pr.nu * k2;
      double2* out = mean ? X + 2 * NK : SC(S3_ETA);   // W, or eta
      lane_qt_solve(N, p, alpha, R2, out, T(1, 0), T(1, 1), T(1, 2), G(1), w1, w2, w3, 0.0, 1.0);
    }
  }
  __syncthreads();
  // phase 6: u, w from D v and eta (k != 0): the derivative on warp 0, the
  // element-wise part over all warps
  const bool dvw = act && !mean;
  if (warp == 0 && dvw) lane_cheb_deriv(X + NK, SC(S3_DVN), N, p);
  __syncthreads();
  if (dvw) {
    const double2* __restrict__ dv = SC(S3_DVN);
    const double2* __restrict__ et = SC(S3_ETA);
    double2* __restrict__ u = X;
    double2* __restrict__ w = X + 2 * NK;
    const double ik2 = 1.0 / k2;
    for (int i = e0; i < e1; ++i) {
      const int n = p + 2 * i;
      u[n] = cscl(mul_i(csub(cscl(dv[n], kx), cscl(et[n], kz))), ik2);
      w[n] = cscl(mul_i(cadd(cscl(dv[n], kz), cscl(et[n], kx))), ik2);
    }
  }
}

__global__ void k_tick3(GroupDev g) {
  const int b = threadIdx.x + blockIdx.x * blockDim.x;
  if (b < g.nb && !g.status[b]) g.count[b] += 1;
}

// ------------------------------------------------------------ diagnostics
// Tile slots: P_E a double; P_MIN, P_MAX keys (dkey) of Tr c; P_AMAX the
// bits of max |Tr c|; P_BAD and the counts 64-bit integers; P_MS the
// mid-plane power sums (doubles, in the first mid_tiles tiles only).
enum { P_E = 0, P_MIN, P_MAX, P_AMAX, P_BAD, P_C3, P_C0, P_B3, P_B0,
       P_MC3, P_MC0, P_MB3, P_MB0, P_MS = 16 /* 8 quantities x 4 powers */ };
constexpr int kMidLanes3 = 8, kMidModesPerBlock3 = 256 / kMidLanes3;   // k_diag_mid3
constexpr int kMidTilePts = 2048;   // mid-plane points per tile of k_diag_count3

__device__ __forceinline__ long long* islots3(double* pp) { return reinterpret_cast<long long*>(pp); }
__device__ __forceinline__ const long long* islots3(const double* pp) {
  return reinterpret_cast<const long long*>(pp);
}
__device__ __forceinline__ bool nonfinite3(double x) {
  return (__double_as_longlong(x) & 0x7ff0000000000000LL) == 0x7ff0000000000000LL;
}
// mid-plane points per tile (at least kMidTilePts, and all npl points within
// the ntile tiles) and the number of tiles that carry them
__device__ __forceinline__ int mid_per(int npl, int ntile) {
  return max(kMidTilePts, (npl + ntile - 1) / ntile);
}
__device__ __forceinline__ int mid_tiles(int npl, int ntile) {
  const int per = mid_per(npl, ntile);
  return (npl + per - 1) / per;
}

// Energy (Fejer in y, Parseval in x and z), extrema of Tr c on the unpadded
// grid, non-finite test; ntile blocks per member.
__global__ void __launch_bounds__(256) k_diag_part3(GroupDev g) {
  const int b = blockIdx.y, tile = blockIdx.x;
  if (g.status[b]) return;
  const int KZ = g.KZ, N = g.N, nx = g.nx, nz = g.nz, Je = g.Me;
  const size_t NK = (size_t)N * KZ;
  const double2* DY = g.DY + (size_t)b * 3 * Je * KZ;
  double e = 0.0;
  KeyExt ext = keyext_empty();
  int bad = 0;
  {
    // modes mx > 0 count twice (Parseval over +-kx)
    const unsigned tot = (unsigned)Je * KZ, per = (tot + g.ntile - 1) / g.ntile;
    const unsigned i0 = tile * per, i1 = min(tot, i0 + per);
    const FastDiv dKZ = fast_div((unsigned)KZ);
    double e0 = 0.0, e1 = 0.0;
    for (unsigned i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      const unsigned j = fdiv(i, dKZ), md = i - j * KZ;
      const double2 a0 = DY[i], a1 = DY[(size_t)Je * KZ + i], a2 = DY[(size_t)2 * Je * KZ + i];
      const double q = fma(a0.x, a0.x, fma(a0.y, a0.y, fma(a1.x, a1.x, fma(a1.y, a1.y,
                           fma(a2.x, a2.x, a2.y * a2.y)))));
      if (md < (unsigned)nz) e0 = fma(g.ccw[j], q, e0);   // mx = 0
      else e1 = fma(g.ccw[j], q, e1);
    }
    e = fma(2.0, e1, e0);
  }
  {
    const double* tr = g.DV + (size_t)b * N * nz * nx;
    const long long tot = (long long)N * nz * nx, per = (tot + g.ntile - 1) / g.ntile;
    const long long i0 = tile * per, i1 = min(tot, i0 + per);
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      const double t = tr[i];
      bad |= nonfinite3(t);
      keyext_add(ext, t);
    }
  }
  {
    const double* Xd = reinterpret_cast<const double*>(g.X + (size_t)b * 9 * NK);
    const long long tot = 18LL * NK, per = (tot + g.ntile - 1) / g.ntile;
    const long long i0 = tile * per, i1 = min(tot, i0 + per);
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) bad |= nonfinite3(Xd[i]);
  }
  __shared__ double sh[32];
  __shared__ long long shk[96];
  e = block_sum(e, sh);
  ext = block_keyext(ext, shk);
  bad = (int)block_isum(bad, shk);
  if (threadIdx.x == 0) {
    double* pp = g.part + ((size_t)b * g.ntile + tile) * kPart;
    pp[P_E] = e;
    islots3(pp)[P_MIN] = ext.mn;
    islots3(pp)[P_MAX] = ext.mx;
    islots3(pp)[P_AMAX] = ext.ma;
    islots3(pp)[P_BAD] = bad ? 1 : 0;
  }
}

// Counts of Tr c < 3, < 0 and the tie bands over the volume (every tile)
// and, in the first mid_tiles tiles, over the (x, z) mid-plane values
// MV[b][8][nz][nx] the same counts and the power sums of the 8 mid-plane
// quantities (histograms too); ntile blocks per member.
__global__ void __launch_bounds__(256) k_diag_count3(GroupDev g) {
  const int b = blockIdx.y, tile = blockIdx.x;
  if (g.status[b]) return;
  const TrBands B = tr_bands(1e-9 * block_tiles_amax(g.part + (size_t)b * g.ntile * kPart, g.ntile, P_AMAX));
  TrCounts c{0, 0, 0, 0}, mc{0, 0, 0, 0};
  {
    const double* tr = g.DV + (size_t)b * g.N * g.nz * g.nx;
    const long long tot = (long long)g.N * g.nz * g.nx, per = (tot + g.ntile - 1) / g.ntile;
    const long long i0 = tile * per, i1 = min(tot, i0 + per);
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) tr_count(c, tr[i], B);
  }
  __shared__ long long shk[32];
  const long long c3 = block_isum(c.c3, shk), c0 = block_isum(c.c0, shk);
  const long long b3 = block_isum(c.b3, shk), b0 = block_isum(c.b0, shk);
  double* pp = g.part + ((size_t)b * g.ntile + tile) * kPart;
  if (threadIdx.x == 0) {
    islots3(pp)[P_C3] = c3; islots3(pp)[P_C0] = c0;
    islots3(pp)[P_B3] = b3; islots3(pp)[P_B0] = b0;
  }
  const int npl = g.nz * g.nx;
  if (tile >= mid_tiles(npl, g.ntile)) return;   // block-uniform
  double sums[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) sums[k] = 0.0;
  {
    const double* MV = g.MV + (size_t)b * 8 * npl;
    const int per = mid_per(npl, g.ntile);
    const int i0 = tile * per, i1 = min(npl, i0 + per);
    const double* hr = g.hrange + (size_t)b * 16;
    unsigned long long* gh = g.hist + (size_t)b * 8 * (PTT_HIST_BINS + 2);
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {   // mid-plane histograms
        const int sl = hist_slot(MV[(size_t)q * npl + i], hr[2 * q], hr[2 * q + 1]);
        if (sl >= 0) atomicAdd(&gh[q * (PTT_HIST_BINS + 2) + sl], 1ULL);
      }
      tr_count(mc, MV[i], B);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const double a = MV[(size_t)q * npl + i], a2 = a * a;
        sums[4 * q] += a; sums[4 * q + 1] += a2; sums[4 * q + 2] += a2 * a; sums[4 * q + 3] += a2 * a2;
      }
    }
  }
  __shared__ double red[8 * 32];
  block_sum_scatter(sums, red);
  const long long m3 = block_isum(mc.c3, shk), m0 = block_isum(mc.c0, shk);
  const long long mb3 = block_isum(mc.b3, shk), mb0 = block_isum(mc.b0, shk);
  if (threadIdx.x < 32) pp[P_MS + threadIdx.x] = red[threadIdx.x];
  if (threadIdx.x == 0) {
    islots3(pp)[P_MC3] = m3; islots3(pp)[P_MC0] = m0;
    islots3(pp)[P_MB3] = mb3; islots3(pp)[P_MB0] = mb0;
  }
}

// Mid-plane spectra at y = 0 per mode (kMidLanes3 lanes each): DM[b][q][mode]
// for q = Tr c, u', w', du/dx, du/dz, dw/dx, dw/dz, v (u', w' without the
// mean).
__device__ __forceinline__ double2 seg_sum2_3(double2 v) {
#pragma unroll
  for (int o = kMidLanes3 / 2; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o, kMidLanes3);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o, kMidLanes3);
  }
  return v;
}
__global__ void __launch_bounds__(256) k_diag_mid3(GroupDev g) {
  const int b = blockIdx.y;
  if (g.status[b]) return;
  const int sub = threadIdx.x & (kMidLanes3 - 1);
  const int md = blockIdx.x * (blockDim.x / kMidLanes3) + (threadIdx.x / kMidLanes3);
  const int KZ = g.KZ, N = g.N, nz = g.nz;
  const bool on = md < KZ;   // every lane takes part in the shuffles
  const size_t NK = (size_t)N * KZ;
  const double2* X = g.X + (size_t)b * 9 * NK + (size_t)(on ? md : 0) * N;
  double2 tr = czero(), u = czero(), v = czero(), w = czero();
  const int r4 = sub & 3;   // n = sub (mod kMidLanes3): one residue of n mod 4 per lane
  if (on && (r4 == 0 || r4 == 2)) {
    const double s = (r4 == 0) ? 1.0 : -1.0;
    for (int n = sub; n < N; n += kMidLanes3) {
      tr = cfma(s, cadd(X[3 * NK + n], cadd(X[6 * NK + n], X[8 * NK + n])), tr);
      u = cfma(s, X[n], u);
      v = cfma(s, X[NK + n], v);
      w = cfma(s, X[2 * NK + n], w);
    }
  }
  tr = seg_sum2_3(tr);
  u = seg_sum2_3(u);
  v = seg_sum2_3(v);
  w = seg_sum2_3(w);
  if (on && sub == 0) {
    const MemberPrm pr = g.prm[b];
    const int mx = md / nz, mzi = md - mx * nz, hz = nz / 2;
    const int sz = (mzi < hz) ? mzi : mzi - nz;
    const double kx = pr.kx1 * mx;
    const double kz = (mzi == hz) ? 0.0 : pr.kz1 * sz;
    double2 q[8] = {tr, u, w, cscl(mul_i(u), kx), cscl(mul_i(u), kz), cscl(mul_i(w), kx),
                    cscl(mul_i(w), kz), v};
    if (md == 0) { q[1] = czero(); q[2] = czero(); }
    double2* D = g.DM + (size_t)b * 8 * KZ + md;
    for (int k = 0; k < 8; ++k) D[(size_t)k * KZ] = q[k];
  }
}

// Per member: reduce the tiles (each thread a fixed set of tiles, then
// fixed-order trees: deterministic; the energy and the mid-plane sums in
// FP64, extrema and counts on integers), <Tr c>, blow-up test, record.
__global__ void __launch_bounds__(256) k_diag_final3(GroupDev g) {
  const int b = blockIdx.x;
  if (g.status[b]) return;
  __shared__ double sh[32];
  __shared__ long long shk[96];
  const int KZ = g.KZ, N = g.N;
  const size_t NK = (size_t)N * KZ;
  const MemberPrm pr = g.prm[b];
  const double* pp = g.part + (size_t)b * g.ntile * kPart;
  const double2* X = g.X + (size_t)b * 9 * NK;
  double mt = 0.0;
  for (int n = threadIdx.x; n < N; n += blockDim.x)
    if ((n & 1) == 0)
      mt += (X[3 * NK + n].x + X[6 * NK + n].x + X[8 * NK + n].x) * (2.0 / (1.0 - (double)n * n));
  mt = block_sum(mt, sh);
  double te = 0.0;
  KeyExt ext = keyext_empty();
  long long tbad = 0, cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int t = threadIdx.x; t < g.ntile; t += blockDim.x) {
    const double* q = pp + (size_t)t * kPart;
    const long long* qi = islots3(q);
    te += q[P_E];
    keyext_merge(ext, KeyExt{qi[P_MIN], qi[P_MAX], qi[P_AMAX]});
    tbad |= qi[P_BAD];
    for (int k = 0; k < 4; ++k) cnt[k] += qi[P_C3 + k];
  }
  const int nmt = mid_tiles(g.nz * g.nx, g.ntile);
  for (int t = threadIdx.x; t < nmt; t += blockDim.x)
    for (int k = 0; k < 4; ++k) cnt[4 + k] += islots3(pp + (size_t)t * kPart)[P_MC3 + k];
  te = block_sum(te, sh);
  ext = block_keyext(ext, shk);
  tbad = block_isum(tbad, shk);
  for (int k = 0; k < 8; ++k) cnt[k] = block_isum(cnt[k], shk);
  // mid-plane sums: thread k < 32 adds slot k over the mid tiles in order
  __shared__ double ms[32];
  if (threadIdx.x < 32) {
    double a = 0.0;
    for (int t = 0; t < nmt; ++t) a += pp[(size_t)t * kPart + P_MS + threadIdx.x];
    ms[threadIdx.x] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double e = 0.25 * te;
    const bool bad = (tbad != 0);
    const long long step = g.count[b];
    const double qnan = __longlong_as_double(0x7ff8000000000000LL);
    ptt_diag& r = g.ring[(size_t)b * kRing + (size_t)(step % kRing)];
    r.step = step;
    r.t = step * pr.dt;
    r.energy = e;
    r.mean_trc = 0.5 * mt;
    r.min_trc = bad ? qnan : dkey_val(ext.mn);
    r.max_trc = bad ? qnan : dkey_val(ext.mx);
    r.n_lt3 = cnt[0]; r.n_lt0 = cnt[1];
    r.n_band3 = cnt[2]; r.n_band0 = cnt[3];
    r.n_mid_lt3 = cnt[4]; r.n_mid_lt0 = cnt[5];
    r.n_mid_band3 = cnt[6]; r.n_mid_band0 = cnt[7];
    for (int q = 0; q < 8; ++q)
      for (int k = 0; k < 4; ++k) r.mid_sums[q][k] = ms[4 * q + k];
    const bool blow = bad || !isfinite(e) || r.max_trc > pr.trc_max || sqrt(2.0 * e) > pr.u_max;
    r.status = blow ? PTT_BLOWUP : PTT_OK;
    r.reserved = 0;
    if (blow) g.status[b] = 1;
    window_add(g.macc + (size_t)b * kMacc, r);
  }
}

__global__ void k_reset3(GroupDev g, int b) {
  if (threadIdx.x == 0) {
    g.count[b] = 0;
    g.status[b] = 0;
  }
}

YJob yjob3(const GroupDev& g, bool inverse, int M, int C, const FftPlan& pl, const double2* tw4) {
  YJob J{};
  J.gauss = tw4 ? 1 : 0;
  J.tw4 = tw4;  // the quarter-period table of this direction
  J.tw4f = inverse ? g.tw4Pif : g.tw4Pf;
  J.tw4d = inverse ? g.tw4Pid : g.tw4Pd;
  J.K = g.KZ;
  J.N = g.N;
  J.M = M;
  J.inverse = inverse ? 1 : 0;
  J.C = C;
  J.pl = pl;
  J.status = g.status;
  J.cm = g.N;
  J.cn = 1;
  J.vm = 1;
  J.vj = g.KZ;
  for (int i = 0; i < kYFields; ++i) J.src_field2[i] = J.src_field3[i] = -1;
  return J;
}

ZJob zjob(const GroupDev& g, bool inverse, int Mz, int rows, const FftPlan& pl) {
  ZJob Z{};
  Z.K = g.K;
  Z.nz = g.nz;
  Z.Mz = Mz;
  Z.inv = 1.0 / Mz;
  Z.invf = (float)Z.inv;
  Z.inverse = inverse ? 1 : 0;
  Z.C = 8;
  Z.rows = rows;
  Z.status = g.status;
  Z.prm = g.prm;
  Z.pl = pl;
  return Z;
}

size_t smem_zcols(int C, int Mz, int f32) { return (size_t)2 * C * Mz * (f32 ? sizeof(float2) : sizeof(double2)); }

template <typename F>
cudaError_t optin3(F* fn, int optin_bytes) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, fn);
  if (e) return e;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin_bytes - (int)a.sharedSizeBytes);
}

}  // namespace

namespace {
constexpr size_t kXfusedSmemMax = 227 * 1024;
}
bool xfused3_inplace(int Mx, int f32) {
  return !f32 && (size_t)36 * Mx * sizeof(double2) > kXfusedSmemMax && Mx <= kIpMaxN;
}
size_t smem_xfused3(int Mx, int f32) {
  const size_t es = f32 ? sizeof(float2) : sizeof(double2);
  const size_t b = (xfused3_inplace(Mx, f32) ? 18 : 36) * (size_t)Mx * es;
  return b <= kXfusedSmemMax ? b : 0;
}
size_t spec3_scratch_columns() { return kScr3; }
size_t smem_zcols3(int C, int Mz, int f32) { return smem_zcols(C, Mz, f32); }

cudaError_t set_kernel_attributes3(int optin_bytes) {
  cudaError_t e;
  if ((e = optin3(k_ycols<double2>, optin_bytes))) return e;
  if ((e = optin3(k_ycols<float2>, optin_bytes))) return e;
  if ((e = optin3(k_ycols<dsc>, optin_bytes))) return e;
  if ((e = optin3(k_zcols<dsc>, optin_bytes))) return e;
  if ((e = optin3(k_xfused3<dsc>, optin_bytes))) return e;
  if ((e = optin3(k_xfused3<dsc, true>, optin_bytes))) return e;
  if ((e = optin3(k_zcols<double2>, optin_bytes))) return e;
  if ((e = optin3(k_zcols<float2>, optin_bytes))) return e;
  if ((e = optin3(k_zcols<double2, true>, optin_bytes))) return e;
  if ((e = optin3(k_zcols<dsc, true>, optin_bytes))) return e;
  if ((e = optin3(k_ycols<dsc, true>, optin_bytes))) return e;
  if ((e = optin3(k_ycols<double2, true>, optin_bytes))) return e;
  if ((e = optin3(k_xfused3<double2>, optin_bytes))) return e;
  if ((e = optin3(k_xfused3<float2>, optin_bytes))) return e;
  if ((e = optin3(k_xfused3<double2, true>, optin_bytes))) return e;
  if ((e = optin3(k_xrows, optin_bytes))) return e;
  return cudaSuccess;
}

static void launch_spec3(const GroupDev& g, int mode, cudaStream_t st) {
  k_spec3<<<dim3(cdiv(g.KZ, kModesPerBlock), g.nb), 256, 0, st>>>(g, mode);
}

// Stage s of one 3D step for one group (same numbering as the 2D stages).
cudaError_t launch_stage3(const GroupDev& g, int stage, cudaStream_t st, int* nl) {
  const int M = g.M, K = g.K, KZ = g.KZ, Mz = g.Mz;
  const size_t NK = (size_t)g.N * KZ;
  const long long yplane = (long long)M * KZ;          // Y3 / V3 field size
  const long long zplane = (long long)M * Mz * K;      // Z3 / W3 field size
  const int f32 = g.f32;
  // element format of the padded-grid intermediates (double-single values
  // in the FP64 arrays of PTT_FP64_DS groups)
  const int fmt = g.ds ? kFmtDS : f32;
  int n = 0;
  switch (stage) {
    case 0: {  // inverse y (17 fields) then inverse z (26 lines)
      YJob J = yjob3(g, true, M, g.Ccol, g.plP, g.tw4Pi);
      J.src = g.X;
      J.dst = f32 ? (void*)g.Y3f : (void*)g.Y3;
      J.dst_f32 = fmt;
      J.src_mstride = 9 * NK; J.dst_mstride = 17 * yplane;
      J.src_fstride = NK; J.dst_fstride = yplane;
      const int sf[17] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 0, 2, 3, 4, 5, 6, 7, 8};
      const int dv[17] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 1, 1};
      const size_t sm = smem_ycols(g.Ccol, M, f32);
      for (int i = 0; i < 17; ++i) { J.src_field[i] = sf[i]; J.dst_field[i] = i; J.deriv[i] = dv[i]; }
      if (f32 && g.ymma) {
        cudaError_t e = launch_cheb_mma(g, true, st, g.nsm);
        if (e) return e;
      } else if (f32) {
        k_ycols<float2><<<dim3(cdiv(KZ, g.Ccol), 17, g.nb), 256, sm, st>>>(J);
      } else if (g.ds) {
        k_ycols<dsc><<<dim3(cdiv(KZ, g.Ccol), 17, g.nb), 256, sm, st>>>(J);
      } else {
        k_ycols<double2><<<dim3(cdiv(KZ, g.Ccol), 17, g.nb), 256, sm, st>>>(J);
      }
      ++n;
      if (f32) {   // the mean column (kx = kz = 0) in double-single, FP64 out
        YJob Jm = J;
        Jm.K = 1; Jm.C = 1; Jm.pl = g.plPn;
        Jm.dst = g.Ym; Jm.dst_f32 = 0;
        Jm.dst_mstride = 17LL * M; Jm.dst_fstride = M;
        Jm.vm = 1; Jm.vj = 1;
        k_ycols<dsc><<<dim3(1, 17, g.nb), 256, smem_ycols(1, M, 0), st>>>(Jm);
        ++n;
      }
      ZJob Z = zjob(g, true, Mz, M, g.plMz);
      Z.C = g.zC;
      Z.src = J.dst; Z.src_f32 = fmt;
      Z.dst = f32 ? (void*)g.Z3f : (void*)g.Z3; Z.dst_f32 = fmt;
      Z.mean = f32 ? 1 : 0;
      Z.src_mstride = 17 * yplane; Z.dst_mstride = 26 * zplane;
      Z.src_fstride = yplane; Z.dst_fstride = zplane;
      for (int i = 0; i < 26; ++i) {
        Z.src_field[i] = (i < 17) ? i : i - 17;
        Z.dst_field[i] = i;
        Z.dz[i] = (i >= 17) ? 1 : 0;
      }
      const size_t smz = smem_zcols(Z.C, Mz, f32);
      if (f32) k_zcols<float2><<<dim3(cdiv(K, Z.C), 26 * M, g.nb), 256, smz, st>>>(Z);
      else if (g.ds) k_zcols<dsc><<<dim3(cdiv(K, Z.C), 26 * M, g.nb), 256, smz, st>>>(Z);
      else k_zcols<double2><<<dim3(cdiv(K, Z.C), 26 * M, g.nb), 256, smz, st>>>(Z);
      ++n;
      break;
    }
    case 1:
      if (f32) k_xfused3<float2><<<dim3(M * Mz, g.nb), g.xthreads, smem_xfused3(g.Mx, 1), st>>>(g);
      else if (g.ds && xfused3_inplace(g.Mx, 0))
        k_xfused3<dsc, true><<<dim3(M * Mz, g.nb), kIpThreads, smem_xfused3(g.Mx, 0), st>>>(g);
      else if (g.ds) k_xfused3<dsc><<<dim3(M * Mz, g.nb), g.xthreads, smem_xfused3(g.Mx, 0), st>>>(g);
      else if (xfused3_inplace(g.Mx, 0))
        k_xfused3<double2, true><<<dim3(M * Mz, g.nb), kIpThreads, smem_xfused3(g.Mx, 0), st>>>(g);
      else k_xfused3<double2><<<dim3(M * Mz, g.nb), g.xthreads, smem_xfused3(g.Mx, 0), st>>>(g);
      n = 1;
      break;
    case 2: {  // forward z (9) then forward y (9)
      ZJob Z = zjob(g, false, Mz, M, g.plMz);
      Z.C = g.zC;
      Z.src = f32 ? (const void*)g.W3f : (const void*)g.W3; Z.src_f32 = fmt;
      Z.dst = f32 ? (void*)g.V3f : (void*)g.V3; Z.dst_f32 = fmt;
      Z.mean = f32 ? 2 : 0;
      Z.zm = g.Zm;
      Z.src_mstride = 9 * zplane; Z.dst_mstride = 9 * yplane;
      Z.src_fstride = zplane; Z.dst_fstride = yplane;
      for (int i = 0; i < 9; ++i) { Z.src_field[i] = i; Z.dst_field[i] = i; Z.dz[i] = 0; }
      const size_t smz = smem_zcols(Z.C, Mz, f32);
      if (f32) k_zcols<float2><<<dim3(cdiv(K, Z.C), 9 * M, g.nb), 256, smz, st>>>(Z);
      else if (g.ds) k_zcols<dsc><<<dim3(cdiv(K, Z.C), 9 * M, g.nb), 256, smz, st>>>(Z);
      else k_zcols<double2><<<dim3(cdiv(K, Z.C), 9 * M, g.nb), 256, smz, st>>>(Z);
      YJob F = yjob3(g, false, M, g.Ccol, g.plP, g.tw4P);
      F.src = Z.dst; F.src_f32 = fmt;
      F.dst = g.NR;
      F.src_mstride = 9 * yplane; F.dst_mstride = 9 * NK;
      F.src_fstride = yplane; F.dst_fstride = NK;
      const size_t sm = smem_ycols(g.Ccol, M, f32);
      for (int i = 0; i < 9; ++i) { F.src_field[i] = i; F.dst_field[i] = i; F.deriv[i] = 0; }
      if (f32 && g.ymma) {
        cudaError_t e = launch_cheb_mma(g, false, st, g.nsm);
        if (e) return e;
      } else if (f32) {
        k_ycols<float2><<<dim3(cdiv(KZ, g.Ccol), 9, g.nb), 256, sm, st>>>(F);
      } else if (g.ds) {
        k_ycols<dsc><<<dim3(cdiv(KZ, g.Ccol), 9, g.nb), 256, sm, st>>>(F);
      } else {
        k_ycols<double2><<<dim3(cdiv(KZ, g.Ccol), 9, g.nb), 256, sm, st>>>(F);
      }
      n = 2;
      if (f32) {   // the mean column in double-single, over the FP32 pass's zeros
        YJob Fm = F;
        Fm.K = 1; Fm.C = 1; Fm.pl = g.plPn;
        Fm.src = g.Zm; Fm.src_f32 = 0;
        Fm.src_mstride = 9LL * M; Fm.src_fstride = M;
        Fm.vm = 1; Fm.vj = 1;
        k_ycols<dsc><<<dim3(1, 9, g.nb), 256, smem_ycols(1, M, 0), st>>>(Fm);
        ++n;
      }
      break;
    }
    case 3:
      launch_spec3(g, 0, st);
      k_tick3<<<cdiv(g.nb, 128), 128, 0, st>>>(g);
      n = 2;
      break;
    case 4: {  // diagnostics, in order on one stream
      const DiagStreams d{{st, st, st}, {nullptr, nullptr, nullptr}};
      return launch_diag_split3(g, d, nl);
    }
    default:
      return cudaErrorInvalidValue;
  }
  if (nl) *nl += n;
  return cudaGetLastError();
}

// Fork d.s[1], d.s[2] off d.s[0] (when distinct) before the parts, join after.
static cudaError_t diag_fork3(const DiagStreams& d) {
  if (d.s[1] == d.s[0]) return cudaSuccess;
  cudaError_t e = cudaEventRecord(d.ev[0], d.s[0]);
  if (!e) e = cudaStreamWaitEvent(d.s[1], d.ev[0], 0);
  if (!e) e = cudaStreamWaitEvent(d.s[2], d.ev[0], 0);
  return e;
}
static cudaError_t diag_join3(const DiagStreams& d) {
  if (d.s[1] == d.s[0]) return cudaSuccess;
  cudaError_t e = cudaEventRecord(d.ev[1], d.s[1]);
  if (!e) e = cudaEventRecord(d.ev[2], d.s[2]);
  if (!e) e = cudaStreamWaitEvent(d.s[0], d.ev[1], 0);
  if (!e) e = cudaStreamWaitEvent(d.s[0], d.ev[2], 0);
  return e;
}

// The diagnostics' y transforms (they write only DY, DT): u, v, w on the Me
// Gauss points; c_xx + c_yy + c_zz on the unpadded Gauss-Lobatto rows.
static void diag_energy_y3(const GroupDev& g, cudaStream_t st) {
  const int KZ = g.KZ;
  const size_t NK = (size_t)g.N * KZ;
  YJob J = yjob3(g, true, g.Me, g.CcolE, g.plPe, g.tw4E);
  J.tw4f = g.tw4Ef;   // mixed groups transform in FP32 (the sums stay FP64)
  J.tw4d = g.tw4Ed;   // double-single groups in double-single
  J.src = g.X; J.dst = g.DY;
  J.src_mstride = 9 * NK; J.dst_mstride = 3LL * g.Me * KZ;
  J.src_fstride = NK; J.dst_fstride = (long long)g.Me * KZ;
  for (int i = 0; i < 3; ++i) { J.src_field[i] = i; J.dst_field[i] = i; J.deriv[i] = 0; }
  if (g.f32) k_ycols<float2><<<dim3(cdiv(KZ, g.CcolE), 3, g.nb), 256, smem_ycols(g.CcolE, g.Me, 1), st>>>(J);
  else if (g.ds) k_ycols<dsc><<<dim3(cdiv(KZ, g.CcolE), 3, g.nb), 256, smem_ycols(g.CcolE, g.Me, 0), st>>>(J);
  else k_ycols<double2><<<dim3(cdiv(KZ, g.CcolE), 3, g.nb), 256, smem_ycols(g.CcolE, g.Me, 0), st>>>(J);
}
static void diag_trc_y3(const GroupDev& g, cudaStream_t st) {
  const int KZ = g.KZ;
  const size_t NK = (size_t)g.N * KZ;
  YJob T = yjob3(g, true, g.N - 1, g.CcolU, g.plPu, nullptr);
  T.src = g.X; T.dst = g.DT;
  T.src_mstride = 9 * NK; T.dst_mstride = (long long)NK;
  T.src_fstride = NK; T.dst_fstride = 0;
  T.src_field[0] = 3; T.src_field2[0] = 6; T.src_field3[0] = 8; T.dst_field[0] = 0; T.deriv[0] = 0;
  if (g.ds || g.f32)   // double-single (FP64 in and out, FP64 sums downstream)
    k_ycols<dsc, true><<<dim3(cdiv(KZ, g.CcolU), 1, g.nb), 256, smem_ycols(g.CcolU, g.Pu, 0), st>>>(T);
  else k_ycols<double2, true><<<dim3(cdiv(KZ, g.CcolU), 1, g.nb), 256, smem_ycols(g.CcolU, g.Pu, 0), st>>>(T);
}

cudaError_t launch_diag_transforms3(const GroupDev& g, cudaStream_t st) {
  diag_energy_y3(g, st);
  diag_trc_y3(g, st);
  return cudaGetLastError();
}

cudaError_t launch_diag_split3(const GroupDev& g, const DiagStreams& d, int* nl) {
  const int KZ = g.KZ, K = g.K;
  const size_t NK = (size_t)g.N * KZ;
  cudaError_t e = diag_fork3(d);
  if (e) return e;
  diag_energy_y3(g, d.s[1]);
  // mid-plane: per-mode sums, then z and x syntheses of the 8 quantities
  k_diag_mid3<<<dim3(cdiv(KZ, kMidModesPerBlock3), g.nb), 256, 0, d.s[2]>>>(g);
  ZJob Zm = zjob(g, true, g.nz, 1, g.plNz);
  Zm.src = g.DM; Zm.src_f32 = 0; Zm.dst = g.DMZ; Zm.dst_f32 = 0;
  Zm.src_mstride = 8LL * KZ; Zm.dst_mstride = 8LL * g.nz * K;
  Zm.src_fstride = KZ; Zm.dst_fstride = (long long)g.nz * K;
  for (int i = 0; i < 8; ++i) { Zm.src_field[i] = i; Zm.dst_field[i] = i; Zm.dz[i] = 0; }
  if (g.ds || g.f32)
    k_zcols<dsc, true><<<dim3(cdiv(K, Zm.C), 8, g.nb), 256, smem_zcols(Zm.C, g.nz, 0), d.s[2]>>>(Zm);
  else k_zcols<double2, true><<<dim3(cdiv(K, Zm.C), 8, g.nb), 256, smem_zcols(Zm.C, g.nz, 0), d.s[2]>>>(Zm);
  XJob Xm{};
  Xm.srcC = g.DMZ; Xm.dstR = g.MV;
  Xm.src_mstride = 8LL * g.nz * K; Xm.dst_mstride = 8LL * g.nz * g.nx;
  Xm.src_fstride = (long long)g.nz * K; Xm.dst_fstride = (long long)g.nz * g.nx;
  Xm.src_rstep = 1; Xm.dst_rstep = 1;
  Xm.nf = 8; Xm.K = K; Xm.n = g.nx; Xm.c2r = 1; Xm.status = g.status; Xm.pl = g.plNx;
  k_xrows<<<dim3(g.nz, g.nb), 256, smem_xrows(4, g.nx), d.s[2]>>>(Xm);
  // Tr c = c_xx + c_yy + c_zz on the unpadded grid: y (Gauss-Lobatto) -> z -> x
  diag_trc_y3(g, d.s[0]);
  ZJob Z = zjob(g, true, g.nz, g.N, g.plNz);
  Z.src = g.DT; Z.src_f32 = 0; Z.dst = g.DZ; Z.dst_f32 = 0;
  Z.src_mstride = (long long)NK; Z.dst_mstride = (long long)g.N * g.nz * K;
  Z.src_fstride = 0; Z.dst_fstride = 0;
  Z.src_field[0] = 0; Z.dst_field[0] = 0; Z.dz[0] = 0;
  if (g.ds || g.f32)
    k_zcols<dsc, true><<<dim3(cdiv(K, Z.C), g.N, g.nb), 256, smem_zcols(Z.C, g.nz, 0), d.s[0]>>>(Z);
  else k_zcols<double2, true><<<dim3(cdiv(K, Z.C), g.N, g.nb), 256, smem_zcols(Z.C, g.nz, 0), d.s[0]>>>(Z);
  XJob X{};
  X.srcC = g.DZ; X.dstR = g.DV;
  X.src_mstride = (long long)g.N * g.nz * K; X.dst_mstride = (long long)g.N * g.nz * g.nx;
  X.src_fstride = 0; X.dst_fstride = 0;
  X.src_rstep = 1; X.dst_rstep = 1;
  X.nf = 1; X.K = K; X.n = g.nx; X.c2r = 1; X.status = g.status; X.pl = g.plNx;
  X.pair_rows = 1; X.nrows = g.N * g.nz;
  k_xrows<<<dim3(cdiv(g.N * g.nz, 2), g.nb), 256, smem_xrows(1, g.nx), d.s[0]>>>(X);
  if ((e = cudaGetLastError()) || (e = diag_join3(d))) return e;
  k_diag_part3<<<dim3(g.ntile, g.nb), 256, 0, d.s[0]>>>(g);
  k_diag_count3<<<dim3(g.ntile, g.nb), 256, 0, d.s[0]>>>(g);
  k_diag_final3<<<g.nb, 256, 0, d.s[0]>>>(g);
  if (nl) *nl += 10;
  return cudaGetLastError();
}

cudaError_t launch_step3(const GroupDev& g, cudaStream_t st, int* nl) {
  for (int s = 0; s < 4; ++s) {
    cudaError_t e = launch_stage3(g, s, st, nl);
    if (e) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_diag3(const GroupDev& g, cudaStream_t st, int* nl) { return launch_stage3(g, 4, st, nl); }

cudaError_t launch_explicit3(const GroupDev& g, cudaStream_t st) {
  for (int s = 0; s < 3; ++s) {
    cudaError_t e = launch_stage3(g, s, st, nullptr);
    if (e) return e;
  }
  launch_spec3(g, 1, st);
  return cudaGetLastError();
}

cudaError_t launch_reset_member3(const GroupDev& g, int b, cudaStream_t st) {
  k_reset3<<<1, 32, 0, st>>>(g, b);
  return cudaGetLastError();
}

// physical staging [9][ny][nz][nx] -> state of member b: x analysis per
// (y, z) row, z analysis per (y, mx), y analysis (DCT-I) per mode.
cudaError_t launch_phys_to_state3(const GroupDev& g, int b, cudaStream_t st) {
  const int K = g.K, KZ = g.KZ, N = g.N, nz = g.nz, nx = g.nx;
  const size_t NK = (size_t)N * KZ;
  const long long rowsp = (long long)N * nz;
  XJob X{};
  X.srcR = g.stage; X.dstC = g.DZ;   // DZ reused as [9][N][nz][K]
  X.src_fstride = rowsp * nx; X.dst_fstride = rowsp * K;
  X.src_rstep = 1; X.dst_rstep = 1;
  X.nf = 9; X.K = K; X.n = nx; X.c2r = 0; X.status = nullptr; X.pl = g.plNx;
  k_xrows<<<dim3((unsigned)rowsp, 1), 256, smem_xrows(5, nx), st>>>(X);
  ZJob Z = zjob(g, false, nz, N, g.plNz);
  Z.status = nullptr;
  Z.src = g.DZ; Z.dst = g.stageS;     // stageS reused as [9][N][KZ]
  Z.src_fstride = rowsp * K; Z.dst_fstride = (long long)N * KZ;
  for (int i = 0; i < 9; ++i) { Z.src_field[i] = i; Z.dst_field[i] = i; Z.dz[i] = 0; }
  k_zcols<double2, true><<<dim3(cdiv(K, Z.C), 9 * N, 1), 256, smem_zcols(Z.C, nz, 0), st>>>(Z);
  YJob J = yjob3(g, false, N - 1, g.CcolU, g.plPu, nullptr);
  J.status = nullptr;
  J.src = g.stageS; J.dst = g.X + (size_t)b * 9 * NK;
  J.src_fstride = (long long)N * KZ; J.dst_fstride = NK;
  for (int i = 0; i < 9; ++i) { J.src_field[i] = i; J.dst_field[i] = i; J.deriv[i] = 0; }
  k_ycols<double2, true><<<dim3(cdiv(KZ, g.CcolU), 9, 1), 256, smem_ycols(g.CcolU, g.Pu, 0), st>>>(J);
  k_reset3<<<1, 32, 0, st>>>(g, b);
  return cudaGetLastError();
}

cudaError_t launch_state_to_phys3(const GroupDev& g, int b, cudaStream_t st) {
  const int K = g.K, KZ = g.KZ, N = g.N, nz = g.nz, nx = g.nx;
  const size_t NK = (size_t)N * KZ;
  const long long rowsp = (long long)N * nz;
  YJob J = yjob3(g, true, N - 1, g.CcolU, g.plPu, nullptr);
  J.status = nullptr;
  J.src = g.X + (size_t)b * 9 * NK; J.dst = g.stageS;
  J.src_fstride = NK; J.dst_fstride = (long long)N * KZ;
  for (int i = 0; i < 9; ++i) { J.src_field[i] = i; J.dst_field[i] = i; J.deriv[i] = 0; }
  k_ycols<double2, true><<<dim3(cdiv(KZ, g.CcolU), 9, 1), 256, smem_ycols(g.CcolU, g.Pu, 0), st>>>(J);
  ZJob Z = zjob(g, true, nz, N, g.plNz);
  Z.status = nullptr;
  Z.src = g.stageS; Z.dst = g.DZ;
  Z.src_fstride = (long long)N * KZ; Z.dst_fstride = rowsp * K;
  for (int i = 0; i < 9; ++i) { Z.src_field[i] = i; Z.dst_field[i] = i; Z.dz[i] = 0; }
  k_zcols<double2, true><<<dim3(cdiv(K, Z.C), 9 * N, 1), 256, smem_zcols(Z.C, nz, 0), st>>>(Z);
  XJob X{};
  X.srcC = g.DZ; X.dstR = g.stage;
  X.src_fstride = rowsp * K; X.dst_fstride = rowsp * nx;
  X.src_rstep = 1; X.dst_rstep = 1;
  X.nf = 9; X.K = K; X.n = nx; X.c2r = 1; X.status = nullptr; X.pl = g.plNx;
  k_xrows<<<dim3((unsigned)rowsp, 1), 256, smem_xrows(5, nx), st>>>(X);
  return cudaGetLastError();
}

}  // namespace ptt
