// Internal declarations shared by the host (C ABI) and device code of the
// sPTT channel library.  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "ptt.h"

namespace ptt {

constexpr int kMaxStages = 16;
constexpr int kRing = 1024;       // diagnostics records kept per member
constexpr int kNumHist = 4;       // SBDF4 history depth

// Mixed-radix (2, 3, 4, 5, 7, 11, 13) Stockham FFT plan of length n.
struct FftPlan {
  int n;
  int nst;
  int radix[kMaxStages];
  const double2* tw;  // tw[k] = exp(-2 pi i k / n), k < n (device)
  const float2* twf;  // the same in single precision (mixed groups), or null
  const float4* twd;  // the same in double-single, (re.h, re.l, im.h, im.l) with
                      // re = re.h + re.l (PTT_FP64_DS groups), or null
  // Tangent-form twiddles of the FP64 passes s >= 1 of radix 2 to 5 (null:
  // use tw; passes of radix 7, 11, 13 always use tw).  Forward
  // twiddle r of stride index jm:
  //   exp(-2 pi i jm r st / n) = i^k_r cos(t'_r) (1 + i tan(t'_r)), |t'_r| <= pi/4,
  // record jm of pass s at tt[tto[s] + RS jm] (RS = 16 for radix 5, else 6),
  // quadrants k_r packed in tk[toff[s] + jm] (2 bits each).  Records:
  // radix 5 (tan1..tan4, cos4/cos1, cos3/cos2, cos1, cos2, C1 cos1, C2 cos2,
  // C2 cos1, C1 cos2, S1 cos1, S2 cos2, S2 cos1, S1 cos2 with C_q, S_q the
  // cosine and sine of 2 pi q/5); radix 4 (tan1, tan2, tan3, cos1, cos2,
  // cos3/cos1); radix 3 (tan1, tan2, cos1, cos2/cos1, cos1/2,
  // sin(2 pi/3) cos1); radix 2 (tan1, cos1).
  const double* tt;
  const int* tk;
  int toff[kMaxStages];
  int tto[kMaxStages];
  // Per-pass constants (plan_pass_consts): butterflies per line n/R, twiddle
  // stride n/(Ns R), span Ns before the pass, and the multiply-high
  // reciprocals of n/R and Ns (0 for 1), so that a pass divides nothing.
  int pnb[kMaxStages], pst[kMaxStages], pns[kMaxStages];
  unsigned pmb[kMaxStages], pms[kMaxStages];
};
// Fills the per-pass constants of pl from pl.n, pl.nst and pl.radix.
void plan_pass_consts(FftPlan& pl);

// Per-member physics, resident on the device.
struct MemberPrm {
  double lx, lz, re, wi, beta, eps, kappa, dt;
  double inv_wi, gam, nu, forcing;  // 1/Wi, (1-beta)/(Re Wi), beta/Re, 2/Re
  double trc_max, u_max;
  // 2 pi / Lx, 2 pi / Lz and their FP32 roundings, computed on the host: a
  // division per thread would cost the FP32 kernels tens of FP64 operations
  double kx1, kz1;
  float kx1f, kz1f;
  float epsf, inv_wif;              // FP32 roundings of eps, 1/Wi
};
// Fills every field of q from p (lz = 1 in 2D).
void member_prm(const ptt_params& p, MemberPrm& q);
// A host-computed constant in the compute precision T: d, or its FP32
// rounding f (no FP64 arithmetic or conversion in the FP32 kernels).
template <typename T> __host__ __device__ __forceinline__ T as_prec(double d, float f);
template <> __host__ __device__ __forceinline__ double as_prec<double>(double d, float) { return d; }
template <> __host__ __device__ __forceinline__ float as_prec<float>(double, float f) { return f; }

// Device view of one group: nb members with equal (nx, ny).
// Spectral arrays are [member][field][m][n] (n fastest), complex double;
// arrays of values on a y grid are [member][field][j][m] (m fastest).
struct GroupDev {
  int nb;            // members in the group
  int ntile;         // diagnostics tiles per member (diag_tiles)
  int xthreads;      // threads per block of the fused x kernels (ptt_autotune)
  int zC;            // 3D: x-mode lines per block of the z passes (ptt_autotune)
  int f32;           // 1: mixed precision (FP32 transforms and products)
  int ds;            // 1: FP64-accurate transforms and products in double-single
                     //    arithmetic on the FP32 pipe (PTT_FP64_DS); the arrays are
                     //    those of an FP64 group, the padded-grid intermediates
                     //    holding double-single values
  int nx, K, N;      // Fourier points / modes (K = nx/2), Chebyshev modes
  int nz, Mz, KZ;    // z modes (1 in 2D), padded z points, modes per Chebyshev index (K * nz)
  double invMx;      // 1 / Mx (host-computed), and its FP32 rounding
  float invMxf;
  int Mx, M, P;      // padded x points, padded y Gauss points (= y FFT length), P = M
  int Pu, Me;        // y FFT length of the unpadded grid (2(N-1)); diagnostic Gauss points
  int Ccol, CcolE, CcolU;  // columns per block: padded / diagnostic / unpadded y passes
  MemberPrm* prm;    // [nb]
  int* status;       // [nb]  0 = running, 1 = blown up
  long long* count;  // [nb]  steps since the state was set
  double2* X;        // [nb][5][K][N]  state u, v, cxx, cxy, cyy
  double2* Eh;       // [4 slot][nb][4][K][N]  evolved quantities (cxx, cxy, cyy, q)
  double2* Nh;       // [4 slot][nb][4][K][N]  their explicit terms
  double2* Yp;       // [nb][9][M][K]  fields on the padded y grid (Gauss points)
  double2* Zp;       // [nb][5][M][K]  products, x-analysed, on the padded y grid
  float2* Ypf;       // mixed groups: Yp in single precision
  float2* Zpf;       // mixed groups: Zp in single precision
  // 3D: [nb][17][M][KZ], [nb][26][M][Mz][K], [nb][9][M][Mz][K], [nb][9][M][KZ]
  double2 *Y3, *Z3, *W3, *V3;
  float2 *Y3f, *Z3f, *W3f, *V3f;
  double2* DZ;       // 3D: Tr c after z synthesis [nb][N][nz][K]; state staging [9][N][nz][K]
  double2* DMZ;      // 3D: mid-plane quantities after z synthesis [nb][8][nz][K]
  double* MV;        // 3D: mid-plane values [nb][8][nz][nx]
  // mixed groups, mean/fluctuation split of the products: the mean Fourier
  // column (kx = 0, and kz = 0 in 3D) of the inverse y pass on the padded
  // Gauss grid, in FP64 ([nb][9][M] in 2D, [nb][17][M] in 3D; the FP32
  // arrays then carry the fluctuations only), and the mean column of the
  // explicit terms on that grid ([nb][5][M], [nb][9][M]); complex like the
  // other columns of the y passes (their imaginary parts are zero)
  double2* Ym;
  double2* Zm;
  double2* NR;       // [nb][5][K][N]  explicit nonlinear terms, spectral
  double2* Rb;       // [nb][4][K][N]  H_x, H_y of ptt_explicit_rhs
  double2* SS;       // 3D: [nb][columns][KZ][N]  per-mode scratch of the spectral stage
  const double* qt;  // [nb][4 order][3 sys][3 (Q, inv, F)][K][N]
  const double* qtG; // [nb][4][3][2 parity][K]
  const double* vh;  // [nb][4][K][N]  homogeneous v of the influence step
  const double* vhS; // [nb][4][2][K]  1 / sum_n n^2 vh_n per parity
  const double* wrow;// [3][N]  1/(4n(n-1)), 1/(2(n^2-1)), 1/(4n(n+1))
  const double* ccw; // [Me] Fejer weights of the diagnostic Gauss grid
  double2* DY;       // [nb][2][Me][K]  u, v on the diagnostic y grid
  double2* DT;       // [nb][N][K]  cxx+cyy on the unpadded y rows, Fourier modes
  double* DV;        // [nb][N][nx]  cxx+cyy on the unpadded grid
  double* part;      // [nb][ntile][kPart]  partial reductions
  double2* DM;       // [nb][4][K]  mid-plane Chebyshev sums per Fourier mode
  ptt_diag* ring;    // [nb][kRing]
  unsigned long long* hist;  // [nb][8][PTT_HIST_BINS + 2] mid-plane histograms
  const double* hrange;      // [nb][8][2] (lo, hi); lo >= hi: quantity off
  // mixed groups: the Chebyshev passes of the step as tensor-core contractions
  // (ymma = 1, PTT_MIXED_TC; see ptt_mma.cu) with their pre-sliced BF16
  // tables, inverse and forward, or as FP32 FFTs (ymma = 0, PTT_MIXED)
  int ymma;
  int nsm;           // streaming multiprocessors of the device (persistent grids)
  const uint16_t* Wyi;
  const uint16_t* Wyf;
  int* mma_err;      // set by a tensor-core pass whose bounded wait ran out
  double* macc;      // [nb][kMacc] window sums: mid_sums[8][4] of every record, then the record count
  double* statout;   // [kMacc] results of the window-statistics kernels (one call at a time)
  double* stage;     // [5][N][nx] host<->device staging (one member at a time)
  double2* stageS;   // [5][N][K]  values on the unpadded y grid, x analysed
  // quarter-period twiddles of the Gauss-grid transforms, with the constant
  // factors of each direction folded in:
  const double2* tw4P;   // [M]  forward: (s_k/2) exp(-i pi k/(2M)), s_0 = 1/M, s_k = 2/M
  const float2* tw4Pf;   // the same in single precision (mixed groups)
  const double2* tw4Pi;  // [M]  inverse: (1/2) exp(+i pi k/(2M))
  const float2* tw4Pif;  // the same in single precision (mixed groups)
  const double2* tw4E;   // [Me] inverse on the diagnostic Gauss grid: (1/2) exp(+i pi k/(2Me))
  const float2* tw4Ef;   // the same in single precision (mixed groups: FP32 energy transform)
  const float4* tw4Pd;   // double-single forward, inverse and diagnostic tables
  const float4* tw4Pid;  // (PTT_FP64_DS groups)
  const float4* tw4Ed;
  FftPlan plP, plMx, plNx, plPu, plPe;   // lengths M, Mx, nx, 2(N-1), Me
  FftPlan plMz, plNz;                    // 3D: lengths Mz, nz
  FftPlan plPn;      // mixed groups: length M with radices up to 5 (the
                     // double-single passes of the mean column; plP may
                     // hold radix-8 passes there)
};

constexpr int kPart = 48;  // values per diagnostics tile
constexpr int kMacc = 33;  // window accumulator per member: 8 x 4 power sums + record count

// Adds one diagnostics record's mid-plane power sums to its member's window
// accumulator (called by the thread that writes the record).
__device__ __forceinline__ void window_add(double* acc, const ptt_diag& r) {
  for (int q = 0; q < 8; ++q)
    for (int k = 0; k < 4; ++k) acc[4 * q + k] += r.mid_sums[q][k];
  acc[32] += 1.0;
}

// Diagnostics tiles per member: about 2048 grid points each, so that one
// member alone still spreads over the SMs; a function of the shape only, so
// that a member's diagnostics do not depend on the ensemble around it.
inline int diag_tiles(int N, int nx, int nz) {
  const long long pts = (long long)N * nx * nz;
  long long t = (pts + 2047) / 2048;
  if (t < 1) t = 1;
  if (t > 1024) t = 1024;
  return (int)t;
}

// Launch wrappers (device code in ptt_kernels.cu).  All asynchronous on `st`.
cudaError_t launch_stage(const GroupDev& g, int stage, cudaStream_t st, int* nlaunch);
cudaError_t launch_step(const GroupDev& g, cudaStream_t st, int* nlaunch);
cudaError_t launch_diag(const GroupDev& g, cudaStream_t st, int* nlaunch);

// The diagnostics stage as three independent parts and a reduction: the Tr c
// chain (unpadded y grid, then z and x), the energy transform, the mid-plane
// sums; the reduction (tiles, counts, histograms, record) reads all three.
// s[0] runs the Tr c chain and the reduction; with s[1], s[2] distinct from
// s[0] the other two parts fork onto them (ev[0] forks, ev[1], ev[2] join),
// as branches of a captured graph.
struct DiagStreams {
  cudaStream_t s[3];
  cudaEvent_t ev[3];
};
cudaError_t launch_diag_split(const GroupDev& g, const DiagStreams& d, int* nlaunch);
// Only the diagnostics' two y transforms (energy grid, unpadded grid); they
// write scratch only (for launch-shape timing).
cudaError_t launch_diag_transforms(const GroupDev& g, cudaStream_t st);
cudaError_t launch_explicit(const GroupDev& g, cudaStream_t st);

// One launch per kernel of each stage over all 2D groups of a context (in
// place of one per group): the plan holds the grids of every launch and the
// device copies of the groups and of their transform jobs (in `dev`, at
// least multi2d_bytes(ng) bytes of the workspace, 256-byte aligned).  Groups
// must all be 2D, of one precision, without tensor-core passes, at most
// multi2d_max_groups() of them.  Results are bitwise those of the per-group
// launches (each block computes what the same block of its group's own
// launch computes).
struct Multi2DPlan;
int multi2d_max_groups();
size_t multi2d_bytes(int ng);
Multi2DPlan* multi2d_create(const std::vector<const GroupDev*>& groups, void* dev, cudaStream_t st,
                            cudaError_t* err);
void multi2d_destroy(Multi2DPlan* p);
cudaError_t launch_stage_multi(const Multi2DPlan* p, int stage, cudaStream_t st, int* nlaunch);
cudaError_t launch_diag_multi(const Multi2DPlan* p, const DiagStreams& d, int* nlaunch);
// physical staging [5][N][nx] -> state of member b (resets counter/status)
cudaError_t launch_phys_to_state(const GroupDev& g, int b, cudaStream_t st);
// state of member b -> physical staging [5][N][nx]
cudaError_t launch_state_to_phys(const GroupDev& g, int b, cudaStream_t st);
cudaError_t launch_reset_member(const GroupDev& g, int b, cudaStream_t st);
cudaError_t set_kernel_attributes(int max_dyn_smem);
// state of member bs of group s -> state of member bd of group d, modes
// copied, padded with zeros or truncated (both 2D or both 3D)
cudaError_t launch_resample(const GroupDev& d, int bd, const GroupDev& s, int bs, cudaStream_t st);
// Window moments of member b (mean, standard deviation, skewness, kurtosis
// of each mid-plane quantity, from its accumulator; npoints mid-plane points
// per record) into g.statout[0..31], the record count into g.statout[32].
cudaError_t launch_window_moments(const GroupDev& g, int b, double npoints, cudaStream_t st);
// L1 distance between the normalised mid-plane histograms ha and hb (each
// [8][PTT_HIST_BINS + 2]) of every quantity into out[0..7].
cudaError_t launch_hist_l1(const unsigned long long* ha, const unsigned long long* hb, double* out,
                           cudaStream_t st);
// 3D (ptt_kernels3d.cu)
cudaError_t set_kernel_attributes3(int max_dyn_smem);
cudaError_t launch_stage3(const GroupDev& g, int stage, cudaStream_t st, int* nlaunch);
cudaError_t launch_step3(const GroupDev& g, cudaStream_t st, int* nlaunch);
cudaError_t launch_diag3(const GroupDev& g, cudaStream_t st, int* nlaunch);
cudaError_t launch_diag_split3(const GroupDev& g, const DiagStreams& d, int* nlaunch);
cudaError_t launch_diag_transforms3(const GroupDev& g, cudaStream_t st);
cudaError_t launch_explicit3(const GroupDev& g, cudaStream_t st);
cudaError_t launch_phys_to_state3(const GroupDev& g, int b, cudaStream_t st);
cudaError_t launch_state_to_phys3(const GroupDev& g, int b, cudaStream_t st);
cudaError_t launch_reset_member3(const GroupDev& g, int b, cudaStream_t st);
// Shared memory of the 3D fused x pass: two buffers of 18 lines, or one
// (in-place passes, 512 threads) where two do not fit and one does (FP64,
// Mx <= 768); 0 when neither fits.
size_t smem_xfused3(int Mx, int f32);
bool xfused3_inplace(int Mx, int f32);
size_t spec3_scratch_columns();
size_t smem_zcols3(int C, int Mz, int f32);

// Tensor-core Chebyshev passes of mixed groups (ptt_mma.cu).
bool cheb_mma_supported(int M, int N);
size_t cheb_mma_table_bytes(int M, int N, int inverse);
void cheb_mma_tables(int M, int N, int inverse, std::vector<uint16_t>& out);
cudaError_t set_cheb_mma_attributes(int optin_bytes);
cudaError_t launch_cheb_mma(const GroupDev& g, bool inverse, cudaStream_t st, int sms);

// Host helpers (ptt_capi.cu) used by the workspace-free entry point.
void set_last_error(const char* msg);
// tt[0], tk[0] / tt[1], tk[1]: tangent-form twiddle records of the padded
// Chebyshev and padded x plans (FftPlan::tt, ::tk).
int shape_plan(const ptt_params& p, GroupDev& d, std::vector<double2>& twP,
               std::vector<double2>& twMx, std::vector<double2>& tw4, MemberPrm& prm,
               std::vector<double>* tt, std::vector<int>* tk);

size_t smem_ycols(int C, int P, int f32);
size_t smem_xfused(int Mx, int f32);
size_t smem_xrows(int nl, int n);
size_t smem_spec(int N);
cudaError_t launch_transpose(const double2* src, double2* dst, int nf, int rows, int cols,
                             cudaStream_t st);

}  // namespace ptt
