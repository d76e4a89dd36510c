/*
 * ptt.h -- C ABI of the GB300-native pseudo-spectral time step for a dilute
 * sPTT polymer solution in a plane channel.
 *
 * The method (Sec. 2 of the paper; Eqs. 1-3):
 *   d_t c + u.grad c - (grad u)^T.c - c.(grad u)
 *         = kappa lap c - (c - I)/Wi [1 + eps Tr(c - I)]               (Eq. 1)
 *   d_t u + u.grad u = -grad p + (beta/Re) lap u
 *         + (1 - beta)/(Re Wi) div c + (2/Re) x_hat                      (Eq. 2)
 *   div u = 0                                                            (Eq. 3)
 * periodic in x (and z), no-slip walls at y = +-1, the wall value of c
 * advanced by Eq. 1 with kappa = 0 (Sec. 2, boundary conditions).  Space:
 * Fourier (x) - Chebyshev (y) modes, fully dealiased products (Sec. 2,
 * numerical details).  Time: fourth-order semi-implicit BDF (SBDF4), started
 * with SBDF1-3.  Diagnostics: Tr c admissibility counts, volume averages
 * E = <|u|^2/2> and <Tr c>, and mid-plane statistics (Sec. 3, Eqs. 4-5).
 *
 * Conventions shared by every call
 *  - A "member" is one independent channel run.  A context holds one or more
 *    members (an ensemble); members with equal (nx, ny, nz, precision) are
 *    advanced together by the same kernel launches.
 *  - nz = 1 selects the 2D (z-independent) problem: w = 0 and c_zz = 1
 *    exactly; the five fields are u, v, c_xx, c_xy, c_yy.  nz > 1 selects the
 *    3D problem with nine fields u, v, w, c_xx, c_xy, c_xz, c_yy, c_yz, c_zz.
 *  - nx: even, 8 <= nx <= 512, of the form 2^a 3^b 5^c 7^d 11^e 13^f.  ny
 *    (Chebyshev modes): 9 <= ny <= 513 with ny - 1 of that form.  nz: 1, or
 *    even with 4 <= nz <= 512 and of that form (then lz > 0).  (Every
 *    multiple of 32 from 64 to 512 is admitted, and so is ny = 225.)
 *  - Physical layout (host arrays of ptt_set_state / ptt_get_state):
 *    double[nf][nz][ny][nx] (2D: nf = 5, nz = 1; 3D: nf = 9): field-major,
 *    then z (z_k = k lz/nz), then y (Gauss-Lobatto point
 *    y_l = cos(pi l/(ny-1)), l = 0 is the wall y = +1), then x
 *    (x_j = j lx/nx) fastest.
 *  - Spectral layout (ptt_get_spectral / ptt_set_spectral): 2D
 *    double[5][ny][nx/2][2]; 3D double[9][ny][nx/2][nz][2]: field, Chebyshev
 *    index n, Fourier index m = 0..nx/2-1 (k_m = 2 pi m / lx; the x Nyquist
 *    mode is not stored), in 3D the z index q = 0..nz-1 in FFT order (signed
 *    wavenumber s = q for q < nz/2, q - nz for q > nz/2, k = 2 pi s / lz; the
 *    slot q = nz/2 of the z Nyquist mode is stored and always zero), (re, im).
 *    The m = 0 plane of a real field is Hermitian in q.
 *  - Device memory: the caller allocates ONE device workspace of at least
 *    ptt_workspace_size() bytes (256-byte aligned) and owns it; the library
 *    never allocates or frees device memory.  Host pointers are caller-owned
 *    and only read or written during the call.
 *  - Streams: every device operation of a context runs on the stream given
 *    to ptt_create (a cudaStream_t passed as void*, NULL = legacy default
 *    stream).  Calls on one context are not re-entrant.
 *  - Errors: every call returns PTT_OK (0), a negative error code, or
 *    PTT_BLOWUP (> 0).  Nothing aborts; no exception crosses the ABI.
 */
#ifndef PTT_H
#define PTT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PTT_OK 0
#define PTT_BLOWUP 1       /* a member blew up (see ptt_diag.status)           */
#define PTT_EINVAL (-1)    /* bad argument, size or pointer                      */
#define PTT_ENOMEM (-2)    /* workspace too small                                */
#define PTT_ECUDA (-3)     /* a CUDA runtime call failed                         */
#define PTT_TIMEOUT (-4)   /* a bounded wait expired                             */
#define PTT_ENOTSUP (-5)   /* valid request this library does not implement      */

#define PTT_FP64 0         /* every step of the path in FP64                     */
#define PTT_MIXED 1        /* FP32 Fourier and Chebyshev transforms (FFTs; the
                              Chebyshev ones as DCT-II/III) and the products'
                              fluctuation parts (means and mean products in
                              FP64, the mean column through double-single y
                              passes); in 2D the explicit-term history and
                              its SBDF sum in FP32 (the mean mode's in FP64);
                              FP64 state and its SBDF sum, tau
                              solves and diagnostic sums (the energy's
                              transform in FP32, the Tr c and mid-plane
                              transforms in double-single)                   */
#define PTT_MIXED_TC 2     /* as PTT_MIXED, with the Chebyshev transforms as dense
                              contractions on the tensor cores: BF16 slices of a
                              fixed-point split, FP32 accumulation (FP32 FFTs for
                              the shapes that contraction does not cover,
                              ny > 321); same accuracy as PTT_MIXED, slower on
                              this part at the shapes measured               */
#define PTT_FP64_DS 3      /* FP64-accurate: the Fourier and Chebyshev transforms
                              and the products in double-single arithmetic
                              (each value the unevaluated sum of two FP32
                              numbers, 48 significant bits) on the FP32 pipe;
                              FP64 state, SBDF sums, tau solves and
                              diagnostics.  Holds the FP64 path's bars against
                              the FP64 solution (1e-11 after one step, 1e-9
                              after 100); GB300's FP64 pipe is 1/64 of its
                              FP32 pipe per instruction                      */

/* Physical and numerical parameters of one member.  Defaults (the paper's
 * single fluid, Sec. 2): lx = lz = 10, re = 1e-2, wi = 150, beta = 0.9,
 * eps = 5e-5, kappa = 5e-5, dt = 2.5e-3. */
typedef struct {
  int32_t nx, ny, nz;        /* Fourier modes in x, Chebyshev modes in y, Fourier
                                modes in z (nz = 1: the 2D problem)             */
  int32_t precision;         /* PTT_FP64, PTT_MIXED, PTT_MIXED_TC or PTT_FP64_DS  */
  double lx, lz;             /* periodic lengths (walls at y = +-1)               */
  double re, wi, beta, eps, kappa;
  double dt;                 /* fixed time step                                   */
  double blowup_trc_max;     /* blow-up if max Tr c exceeds this (e.g. 1e10)      */
  double blowup_u_max;       /* blow-up if sqrt(2 E) exceeds this (e.g. 1e3)      */
} ptt_params;

/* One diagnostics record per member and step (Sec. 3).  Counts are over the
 * unpadded grid (nx * ny * nz points) or the mid-plane y = 0 (nx * nz
 * points).  The
 * strict counts are the paper's; the band counts give the points with
 * |Tr c - 3| <= tau (resp. |Tr c| <= tau), tau = 1e-9 max|Tr c|, whose side
 * of the threshold rounding decides. */
typedef struct {
  int64_t step;              /* steps taken since the state was set               */
  double t;                  /* step * dt                                          */
  double energy;             /* E = <|u|^2 / 2>, volume average                   */
  double mean_trc;           /* <Tr c>, volume average                             */
  double min_trc, max_trc;   /* over the unpadded grid                             */
  int64_t n_lt3, n_lt0, n_band3, n_band0;
  int64_t n_mid_lt3, n_mid_lt0, n_mid_band3, n_mid_band0;
  /* mid-plane power sums: mid_sums[q][p-1] = sum over the mid-plane points of
   * q^p, p = 1..4.  2D: q = Tr c, u' = u - <u>_x, v, du/dx, dv/dx, du/dy
   * (slots 6, 7 unused).  3D: q = Tr c, u' = u - <u>_xz, w' = w - <w>_xz,
   * du/dx, du/dz, dw/dx, dw/dz, v. */
  double mid_sums[8][4];
  int32_t status;            /* PTT_OK or PTT_BLOWUP                               */
  int32_t reserved;
} ptt_diag;

typedef struct ptt_ctx ptt_ctx; /* opaque: host metadata and the step graphs, no data */

/* Bytes of device workspace needed by nmembers members with these params
 * (one params struct per member).  Returns PTT_EINVAL / PTT_ENOTSUP for
 * unsupported params. */
int ptt_workspace_size(const ptt_params* per_member, int32_t nmembers, size_t* bytes);

/* Create a context over the caller's workspace.  per_member points to
 * nmembers params structs (members may differ in every field; those with
 * equal nx, ny share launches).  Builds the operator tables on the host and
 * uploads them; the members' states are zero until ptt_init_state /
 * ptt_set_state.  Synchronous. */
int ptt_create(const ptt_params* per_member, int32_t nmembers, void* d_workspace,
               size_t bytes, void* cuda_stream, ptt_ctx** out);

/* The same as ptt_create, under the name for a batched ensemble of runs of
 * uneven shapes and parameters (one params struct per member). */
int ptt_create_ensemble(const ptt_params* per_member, int32_t nmembers, void* d_workspace,
                        size_t bytes, void* cuda_stream, ptt_ctx** out);

/* Laminar sPTT state (the kappa = 0 closed form of Eqs. 1-2 for channel flow)
 * plus a seeded divergence-free, no-slip perturbation of maximum grid
 * amplitude `amplitude`.  2D: stream function (1 - y^2)^2 g(x, y), g with
 * modes 1 <= m <= 4, n <= 8.  3D: u' = d psi1/dy, v' = -d psi1/dx -
 * d psi2/dz, w' = d psi2/dy with psi_c = (1 - y^2)^2 g_c(x, y, z), g_c with
 * 0 <= mx <= 4, 0 <= mz <= 2, (mx, mz) != (0, 0), n <= 8, scaled so that
 * max |u'| over the grid is `amplitude`.  Coefficients are uniform in
 * [-1, 1) from the counter-based splitmix64 stream of `seed`.  The laminar
 * state depends on y alone: c is not perturbed, and its coefficients at
 * nonzero wavenumbers are exactly zero.  Stands in for the paper's turbulent initial snapshot (Sec. 2),
 * which is not available.  Resets the step counter and the SBDF history.
 * Synchronous. */
int ptt_init_state(ptt_ctx* ctx, int32_t member, uint64_t seed, double amplitude);

/* Set / get the state of one member as physical values on the unpadded grid
 * (layout above).  set: interpolates (Fourier analysis without the Nyquist
 * mode, Chebyshev interpolation at the Gauss-Lobatto points), resets the step
 * counter and history.  Synchronous. */
int ptt_set_state(ptt_ctx* ctx, int32_t member, const double* h_phys);
int ptt_get_state(ptt_ctx* ctx, int32_t member, double* h_phys);

/* Spectral coefficients of the current state (layout above).  set resets the
 * step counter and history.  Synchronous. */
int ptt_set_spectral(ptt_ctx* ctx, int32_t member, const double* h_spec);
int ptt_get_spectral(ptt_ctx* ctx, int32_t member, double* h_spec);

/* Spectral re-interpolation (Sec. 2: a snapshot re-interpolated onto the
 * grids of runs at other resolutions).  Sets the state of member dst_member
 * of dst to the current state of member src_member of src, coefficient by
 * coefficient: Fourier modes (kx, and in 3D kz by signed wavenumber) and
 * Chebyshev modes present in both shapes are copied, modes only the
 * destination has are zero, modes only the source has are dropped (the x and
 * z Nyquist slots stay zero).  Both members must be 2D or both 3D; their
 * periodic lengths should agree (not checked).  Both contexts must live on
 * the current device; src and dst may be the same context.  Resets the
 * destination's step counter and SBDF history and writes its diagnostics
 * record, as ptt_set_spectral does.  Synchronous (waits for both streams). */
int ptt_resample(ptt_ctx* dst, int32_t dst_member, ptt_ctx* src, int32_t src_member);

/* Advance every member by nsteps steps (asynchronous on the context stream;
 * nsteps + 1 CUDA-graph launches: each step's diagnostics run beside the next
 * step's transforms, and those of the last step in one more launch).  A
 * member that blows up stops and keeps its last record's status; the others
 * continue.  Returns PTT_OK or an error; blow-up is reported by
 * ptt_synchronize / ptt_diagnostics. */
int ptt_step(ptt_ctx* ctx, int32_t nsteps);

/* Wait for the context stream, polling it (cudaStreamQuery) for at most the
 * context's wall-clock limit (ptt_set_timeout; 3600 s unless set).  Returns
 * PTT_BLOWUP if any member has blown up, PTT_OK otherwise, PTT_TIMEOUT if the
 * limit passed with work still in flight (nothing is cancelled: the work
 * goes on and a later call waits for it again), or PTT_ECUDA. */
int ptt_synchronize(ptt_ctx* ctx);

/* ptt_synchronize with an explicit limit of `seconds` (< 0: no limit; 0:
 * PTT_TIMEOUT at once unless the stream is idle). */
int ptt_synchronize_for(ptt_ctx* ctx, double seconds);

/* Set the wall-clock limit of ptt_synchronize (seconds; <= 0: no limit). */
int ptt_set_timeout(ptt_ctx* ctx, double seconds);

/* Copy out the diagnostics records of `member` written since the previous
 * call (oldest first; at most max_records, the device ring keeps the last
 * 1024 steps).  Synchronous. */
int ptt_diagnostics(ptt_ctx* ctx, int32_t member, ptt_diag* h_out, int32_t max_records,
                    int32_t* n_written);

/* Mid-plane histograms (Sec. 3: the PDFs of Tr c, of the velocity
 * fluctuations and of the velocity gradients at the mid-plane).  For each of
 * the 8 mid-plane quantities of ptt_diag.mid_sums (same order), counts over
 * PTT_HIST_BINS uniform bins on [lo[q], hi[q]): a value x goes to bin
 * 1 + min(floor((x - lo) * (PTT_HIST_BINS / (hi - lo))), PTT_HIST_BINS - 1)
 * (both factors in FP64), to slot 0 if x < lo, to slot PTT_HIST_BINS + 1 if
 * x >= hi or x is not finite.  lo[q] >= hi[q] switches quantity q off.
 * ptt_set_histograms sets the ranges of one member and zeroes its counts;
 * from then on every diagnostics record written for the member (each step,
 * and the record written by ptt_init_state / ptt_set_state /
 * ptt_set_spectral / ptt_set_checkpoint) adds its nx * nz mid-plane values.
 * ptt_get_histograms copies the counts, int64_t[8][PTT_HIST_BINS + 2].
 * Histograms are not part of a checkpoint.  Synchronous. */
#define PTT_HIST_BINS 256
int ptt_set_histograms(ptt_ctx* ctx, int32_t member, const double* lo, const double* hi);
int ptt_get_histograms(ptt_ctx* ctx, int32_t member, int64_t* counts);

/* Window statistics of the mid-plane quantities (Sec. 3: the paper judges
 * runs by the moments and PDFs of the mid-plane Tr c, velocity fluctuations
 * and velocity gradients over a time window).  Every diagnostics record
 * written for a member (each step, and the record written by ptt_init_state
 * / ptt_set_state / ptt_set_spectral / ptt_set_checkpoint) adds its power
 * sums ptt_diag.mid_sums to the member's window accumulator on the device;
 * ptt_reset_moments zeroes it (ptt_create starts it at zero).  The
 * accumulator is not part of a checkpoint.
 * ptt_midplane_moments computes on the device, in FP64, for each of the 8
 * quantities q (order of ptt_diag.mid_sums), with n = nx nz records samples
 * and raw moments m_p = S_p / n of the accumulated sums S_p:
 *   moments[q][0] = mean m_1, moments[q][1] = standard deviation
 *   sd = sqrt(m_2 - m_1^2), moments[q][2] = skewness
 *   (m_3 - 3 m_1 m_2 + 2 m_1^3) / sd^3, moments[q][3] = kurtosis
 *   (m_4 - 4 m_1 m_3 + 6 m_1^2 m_2 - 3 m_1^4) / sd^4
 * (skewness and kurtosis 0 where sd = 0); moments is double[8][4], nrecords
 * (may be NULL) receives the number of records in the window.  The raw-moment
 * form loses relative accuracy in sd when sd is many orders of magnitude
 * below |mean| (about 1e-16 |mean|^2 / sd^2).  Synchronous. */
int ptt_reset_moments(ptt_ctx* ctx, int32_t member);
int ptt_midplane_moments(ptt_ctx* ctx, int32_t member, double* moments, int64_t* nrecords);

/* L1 distance between the mid-plane histograms of two members (of the same
 * or different contexts on the current device), per quantity:
 * l1[q] = sum over the PTT_HIST_BINS + 2 slots of |a_i / A - b_i / B|, A and
 * B the total counts (0: identical PDFs, 2: disjoint; 0 if both are empty and
 * 2 if only one is).  The two histograms should have been set with the same
 * ranges (not checked).  Computed on the device in FP64 on ctx_a's stream
 * after ctx_b's stream is idle; double[8].  Synchronous. */
int ptt_histogram_l1(ptt_ctx* ctx_a, int32_t member_a, ptt_ctx* ctx_b, int32_t member_b,
                     double* l1);

/* Dealiased explicit right-hand side of the current state of one member
 * (Eq. 1 without kappa lap c; Eq. 2 without pressure and viscous terms) in
 * the spectral layout above: 2D N_cxx, N_cxy, N_cyy, H_x, H_y (5 fields);
 * 3D N_cxx, N_cxy, N_cxz, N_cyy, N_cyz, N_czz, H_x, H_y, H_z (9 fields);
 * H_x includes the forcing 2/Re on its mean mode.  Does not advance the
 * state.  Synchronous. */
int ptt_explicit_rhs(ptt_ctx* ctx, int32_t member, double* h_spec);

/* Workspace-free explicit right-hand side, for callers that cannot allocate
 * device memory (an application that owns every device byte and hands this
 * library none, a plugin with no allocator of its own, a loop in which an
 * allocation and its implicit synchronisation are not allowed).  The paper
 * has no counterpart: this is a deployment variant of ptt_explicit_rhs.
 *
 * Same output as ptt_explicit_rhs for one run with params *p, but from and
 * to device memory the caller passes (FP64 2D only: PTT_ENOTSUP for
 * PTT_MIXED or nz > 1): d_spec holds the spectral state
 * double[5][ny][nx/2][2] (u, v, c_xx, c_xy, c_yy), d_out receives
 * double[5][ny][nx/2][2] (N_cxx, N_cxy, N_cyy, H_x, H_y); both 16-byte
 * aligned, distinct.  The intermediates live in a static device array of
 * 48 MiB that the library image carries (held on every GPU that loads the
 * library until the process exits); shapes whose intermediates exceed it
 * ((12 ny + 14 M) (nx/2) 16 bytes plus tables, M the padded Chebyshev
 * grid: every shape up to nx = 512, ny = 257 fits, nx = 512, ny = 513 does
 * not) return PTT_ENOMEM with the sizes in ptt_last_error().  No device
 * memory is allocated or freed.
 *
 * Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress, which allocates nothing) and, the first time an
 * address is seen on a device, sets the kernels' shared-memory limits.  The
 * call copies its tables from host memory and synchronises its stream, so it
 * must not be made while cuda_stream is being captured into a CUDA graph
 * (PTT_EINVAL).  Every call on a device shares the one array and rewrites
 * what it needs (the array keeps the last call's contents), so calls that
 * overlap on the GPU -- from different host threads or streams -- race and
 * must be serialised by the caller.  The kernels and FFT passes are those of
 * ptt_explicit_rhs.  Runs on cuda_stream (a cudaStream_t as void*) and
 * returns after synchronising it. */
int ptt_explicit_rhs_noalloc(const ptt_params* p, const double* d_spec, double* d_out,
                             void* cuda_stream);

/* Checkpoint of one member: state, SBDF history and step counter, so that a
 * restart continues bit for bit.  ptt_checkpoint_size gives the bytes.
 * Synchronous. */
int ptt_checkpoint_size(ptt_ctx* ctx, int32_t member, size_t* bytes);
int ptt_get_checkpoint(ptt_ctx* ctx, int32_t member, void* h_buf, size_t bytes);
int ptt_set_checkpoint(ptt_ctx* ctx, int32_t member, const void* h_buf, size_t bytes);

/* Stages of one step, in launch order: 0 inverse Chebyshev transforms
 * (2D 9 columns, 3D 17, with d/dy; in 3D followed by the inverse z
 * transforms), 1 fused x transforms + products of Eqs. 1-2, 2 forward
 * transforms (3D: z, then Chebyshev; 2D: Chebyshev), 3 per-mode spectral
 * stage (explicit linear terms, SBDF sums, tau solves, velocity from
 * continuity), 4 diagnostics. */
#define PTT_NSTAGES 5

/* Advance every member by nsteps steps with ordinary (non-graph) launches,
 * recording CUDA events on the context stream around each stage, and add the
 * device time of stage s, summed over groups and steps, to ms[s]
 * (milliseconds, s < PTT_NSTAGES; the caller zeroes ms).  Same arithmetic as
 * ptt_step.  Synchronous. */
int ptt_time_stages(ptt_ctx* ctx, int32_t nsteps, double* ms);

/* Algorithmic work of one step of all members, per stage: flops[s] (complex
 * FFT of length n counted 5 n log2 n, products and recurrences by their
 * operation counts), bytes[s] (compulsory device-memory reads + writes of
 * the stage's inputs and outputs), launches[s] (kernel launches). */
int ptt_stage_work(ptt_ctx* ctx, double* flops, double* bytes, int32_t* launches);

/* Launch-shape autotuner.  For every shape group of the context, times
 * (CUDA events, a few launches each) the candidate launch shapes of the
 * transform stages and keeps the fastest: threads per block of the fused x
 * pass (128..512), Chebyshev columns per block of the y passes and of the
 * diagnostics' two y transforms (1..16, as shared memory allows) and, in 3D,
 * x-mode lines per block of the z passes (1..64); then re-captures the step
 * graph.  These launches read the state without changing it (the
 * diagnostics' records and histograms are not touched) and a launch shape
 * changes only which thread computes what, so results are bitwise the same
 * before and after.  choices (may be
 * NULL) receives, per group in creation order (at most max_groups), the
 * chosen (columns, lines, threads); groups are the distinct (nx, ny, nz,
 * precision) of the members in order of first appearance.  Synchronous. */
int ptt_autotune(ptt_ctx* ctx, int32_t* choices, int32_t max_groups);

/* Launch mode of the step graphs.  0 (the default): every shape group of
 * the context is its own branch of the graph, with its own launches.  1: one
 * launch per kernel of each stage over all groups, each group's blocks
 * found from a table of per-group block counts (a work list over (group,
 * block)), so that a step makes the same dozen or so launches however many
 * shape groups the ensemble holds.  Mode 1 needs 2 to 64 groups, all 2D (nz
 * = 1), of one precision and without tensor-core passes (PTT_ENOTSUP
 * otherwise).  The arithmetic of every block is that of the same block of
 * its group's own launch, so states, records and histograms are bitwise the
 * same in both modes.  Re-captures the step graphs.  Synchronous. */
int ptt_set_launch_mode(ptt_ctx* ctx, int32_t mode);

/* Number of kernel launches one step makes (for launch accounting). */
int ptt_launches_per_step(ptt_ctx* ctx, int32_t* n);

/* Release host resources (the workspace stays the caller's). */
int ptt_destroy(ptt_ctx* ctx);

/* Text of the last CUDA failure of this thread (which call, which line,
 * cudaGetErrorString), "" if none.  Static storage, valid until the next
 * failing call on this thread. */
const char* ptt_last_error(void);

/* Static string naming a status code. */
const char* ptt_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* PTT_H */
