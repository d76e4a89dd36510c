// Chebyshev transforms of the mixed-precision step (PTT_MIXED_TC) as dense
// contractions on the tensor cores (tcgen05, sm_103a): BF16 operands, FP32
// accumulation.
//
// Along y the method (Sec. 2: Fourier-Chebyshev pseudo-spectral) maps the
// Chebyshev coefficients a_n (n < N) of every Fourier column to values on the
// padded grid of M Gauss points y_j = cos(theta_j), theta_j = pi (2j+1)/(2M):
//   inverse  f_j  = sum_n T_n(y_j) a_n,          f'_j = sum_n T_n'(y_j) a_n,
//            T_n(y_j) = cos(n theta_j),  T_n'(y_j) = n sin(n theta_j) / sin(theta_j)
//   forward  a_k  = s_k sum_j cos(k theta_j) f_j  (k < N; s_0 = 1/M, s_k = 2/M),
// i.e. one matrix W (M x N, or N x M) applied to every column.  With the
// columns' real and imaginary parts as the rows of the data operand X
// (128 per tile), each transform is OUT[128 x nout] = X[128 x kin] W^T.
//
// Precision (a fixed-point split in the manner of Ozaki's scheme).  Each data
// row r is scaled by a power of two 2^(7 - e_r), 2^e_r > max_i |x_ri|, and cut
// into four slices of integers in [-128, 128]:
//   x 2^(7 - e_r) = X0 + X1/2^8 + X2/2^16 + X3/2^24 + (|rest| <= 2^-25),
// each slice exact in BF16 (8 significant bits).  The tables are cut the same
// way on the host, row o scaled by a power of two sigma_o > max_i |w_oi|
// (W0 .. W3).  Then
//   out = 2^(e_r - 14) sigma_o (A0 + A1/2^8),
//   A0 = sum_i X0 W0                      (|A0| <= 2^14 kin < 2^24: every
//                                          partial sum is an integer held
//                                          exactly in FP32, whatever rounding
//                                          the tensor core's accumulator uses)
//   A1 = sum_i (X0 W1 + X1 W0) + (X0 W2 + X1 W1 + X2 W0)/2^8
//              + (X0 W3 + X1 W2 + X2 W1 + X3 W0)/2^16
// in two FP32 accumulators in tensor memory (the powers of two ride on
// pre-scaled slices, X2/2^8, X3/2^16, W1/2^8, W2/2^8, W2/2^16, W3/2^16, all
// exact in BF16).  The accumulation error of A1 enters 2^-8 smaller, and the
// dropped products are below 2^-31 of each row's scale.  A fourth slice is
// needed because the derivative table grows like n^2 while the coefficients
// decay: a 24-bit cut of the data loses up to 1e-4 of the derivative at
// ny = 257, the 32-bit cut keeps FP32 accuracy.  Each Fourier column is
// scaled by its own largest coefficient, so the fluctuation columns keep
// their own relative accuracy however large the mean column (the base state,
// stretch components 10^4).
//
// Kernel structure (k_cheb_mma): persistent, one CTA of 512 threads per SM,
// walking tiles (member, field, 64 Fourier columns).  Per tile a first pass
// over the input finds each row's exponent; then, per pass (a set of output
// subtiles whose two accumulators fit the 512 tensor-memory columns), the
// contraction runs in chunks of 32 along kin through a two-stage ring in
// shared memory: all threads load the chunk's data (coalesced along the
// input's contiguous direction), slice it and store the slices in the
// canonical K-major layout (core matrices of 8 rows x 16 bytes), while
// thread 0 brings the chunk of the pre-sliced table with bulk copies
// (cp.async.bulk, completion on an mbarrier) and issues the tcgen05.mma
// instructions; tcgen05.commit on a per-stage mbarrier frees the stage.  The
// epilogue reads the accumulators with tcgen05.ld: inverse outputs
// ([j][column], FP32) go straight to global memory, forward outputs
// ([column][k], FP64) through shared memory so that the writes are
// contiguous.  Every wait is bounded; a wait that runs out sets *err and the
// CTA stops after a bounded wait for its own copies.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <type_traits>
#include <vector>

#include "ptt_internal.h"

namespace ptt {

namespace {

constexpr int kThreads = 512;
constexpr int kVals = 4;                   // contraction indices per thread and chunk
constexpr int kRows = 128;                 // data rows per tile (64 complex columns)
constexpr int kCols = 64;                  // complex columns per tile
constexpr int kChunk = 32;                 // contraction elements per chunk (2 MMA k-steps)
constexpr int kPieceA = kRows * kChunk * 2;  // bytes of one BF16 slice of the data chunk
constexpr int kNPA = 4;                    // data slices: X0, X1, X2/2^8, X3/2^16
constexpr int kNPB = 6;                    // table slices: W0, W1, W1/2^8, W2/2^8, W2/2^16, W3/2^16
constexpr int kMaxW = 208;                 // widest output subtile (two stages fit shared memory)
constexpr int kLBO = 128;                  // core-matrix stride along K (bytes)
constexpr int kSBO = 512;                  // core-matrix stride along rows (4 core matrices of K)
constexpr long long kSpin = 1LL << 26;     // iteration limit of every wait
constexpr int kSmemLimit = 227 * 1024 - 6144;  // dynamic shared memory of one CTA (6 KB static)
constexpr int kTmemCols = 512;
constexpr int kMaxUnits = 8;               // (table, subtile) units
constexpr int kMaxPass = 8;

struct MmaJob {
  const void* in;
  void* out;
  long long in_ms, in_fs, in_cs, in_is;    // complex-element strides: member, field, column, index
  long long out_ms, out_fs, out_cs, out_os;
  int in_f64, out_f64;
  int ncol, kin, nout;
  int nkstep, nchunk;  // 16-wide k-steps, 32-wide chunks
  int nopad;           // nout rounded up to 16
  int nunit;           // (table, subtile) units
  int u_tab[kMaxUnits], u_o0[kMaxUnits], u_w[kMaxUnits];
  long long u_goff[kMaxUnits];  // byte offset of the unit's chunk 0 in W (chunk stride kNPB w 64)
  int npass;
  int p_u0[kMaxPass], p_nu[kMaxPass];  // units of each pass
  int nsrc, ntab;
  int dst[2][9];       // output field per (table, source field); -1: none
  const unsigned char* W;   // sliced tables [unit][chunk][slice][w rows x 32 canonical], BF16
  const float* sigma;       // row scales [table][nopad]
  int ntcol;           // column tiles per (member, field)
  long long ntiles;
  const int* status;
  int* err;
  int stage_bytes;     // data slices (kNPA x kPieceA) + the largest pass's table chunk
  int split;           // 1: one work item per (tile, pass)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor: K-major, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)(kLBO >> 4) << 16;
  d |= (uint64_t)(kSBO >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor: BF16 x BF16 -> FP32, both K-major, M = 128.
__device__ __forceinline__ uint32_t umma_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      :: "r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :: "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done = 0;
  for (long long it = 0; it < kSpin && !done; ++it) {
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  }
  return done != 0;
}

// Both accumulators of 16 output columns of this warp's 32 TMEM lanes (one
// wait for the two loads).
__device__ __forceinline__ void tmem_ld16x2(uint32_t ta, uint32_t tb, uint32_t (&r)[16], uint32_t (&s)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(ta));
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(s[0]), "=r"(s[1]), "=r"(s[2]), "=r"(s[3]), "=r"(s[4]), "=r"(s[5]), "=r"(s[6]), "=r"(s[7]),
        "=r"(s[8]), "=r"(s[9]), "=r"(s[10]), "=r"(s[11]), "=r"(s[12]), "=r"(s[13]), "=r"(s[14]), "=r"(s[15])
      : "r"(tb));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// FP64 value of an FP32 one by integer operations (exact for normal values;
// zero and subnormals give a signed zero, infinities stay, NaN is NaN).
__device__ __forceinline__ double f32_to_f64_bits(float v) {
  const uint32_t b = __float_as_uint(v);
  const uint32_t sign = b & 0x80000000u, e = (b >> 23) & 0xFFu, m = b & 0x7FFFFFu;
  unsigned long long r;
  if (e == 0u) r = (unsigned long long)sign << 32;
  else if (e == 255u) r = ((unsigned long long)(sign | 0x7FF00000u | (m ? 0x80000u : 0u))) << 32;
  else r = ((unsigned long long)(sign | ((e + 896u) << 20) | (m >> 3)) << 32) | ((unsigned long long)(m & 7u) << 29);
  return __longlong_as_double((long long)r);
}

// FP32 value of an FP64 one, mantissa truncated, by integer operations (the
// FP64 pipe is slow on this part): zero and values below the FP32 normal
// range give a signed zero, values beyond it infinity, NaN stays NaN.
__device__ __forceinline__ float f64_to_f32_trunc(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const uint32_t hi = (uint32_t)(u >> 32);
  const uint32_t sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FF);
  const uint32_t mant = (uint32_t)((u >> 29) & 0x7FFFFFu);
  const int ef = e - 1023 + 127;
  uint32_t b;
  if (e == 0x7FF) b = sign | 0x7F800000u | (mant ? 0x400000u : 0u);
  else if (ef <= 0) b = sign;
  else if (ef >= 255) b = sign | 0x7F800000u;
  else b = sign | ((uint32_t)ef << 23) | mant;
  return __uint_as_float(b);
}

// Raw input of one thread for one chunk: kVals complex elements of column m
// at contraction indices i0 .. i0 + kVals - 1 (zero outside the field),
// loaded ahead of their use so that the next chunk's loads overlap this
// chunk's work.
template <bool F64> struct Raw;
template <> struct Raw<true> { double2 v[kVals]; };
template <> struct Raw<false> { float2 v[kVals]; };

template <bool F64>
__device__ __forceinline__ void load_raw(const MmaJob& J, const char* inb, int col0, int ncv, int i0, int m,
                                         Raw<F64>& r) {
  using C = decltype(r.v[0]);
  using CT = typename std::remove_reference<C>::type;
  const bool colok = m < ncv;
  const CT* p = reinterpret_cast<const CT*>(inb) + (long long)(col0 + m) * J.in_cs;
#pragma unroll
  for (int e = 0; e < kVals; ++e) {
    const int i = i0 + e;
    CT z{};
    r.v[e] = (colok && i < J.kin) ? __ldg(p + (long long)i * J.in_is) : z;
  }
}

template <bool F64>
__device__ __forceinline__ void raw_values(const Raw<F64>& r, float (&re)[kVals], float (&im)[kVals]) {
#pragma unroll
  for (int e = 0; e < kVals; ++e) {
    if constexpr (F64) {
      re[e] = f64_to_f32_trunc(r.v[e].x);
      im[e] = f64_to_f32_trunc(r.v[e].y);
    } else {
      re[e] = r.v[e].x;
      im[e] = r.v[e].y;
    }
  }
}

// Slices of x scaled by sc (a power of two, |x sc| < 128): X0, X1, X2/2^8
// and X3/2^16, each exact in BF16.  xs - x0 and the later remainders are
// exact in FP32, and so are their products by 256.
__device__ __forceinline__ void slice4(float x, float sc, float (&p)[kNPA]) {
  const float xs = x * sc;
  const float x0 = rintf(xs);
  const float t1 = (xs - x0) * 256.f;
  const float x1 = rintf(t1);
  const float t2 = (t1 - x1) * 256.f;
  const float x2 = rintf(t2);
  const float x3 = rintf((t2 - x2) * 256.f);
  p[0] = x0;
  p[1] = x1;
  p[2] = x2 * (1.f / 256.f);
  p[3] = x3 * (1.f / 65536.f);
}

// Two exact-in-BF16 values as one BF16x2 word (a in the low half).
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
  return r;
}

template <bool F64>
__global__ void __launch_bounds__(kThreads, 1) k_cheb_mma(MmaJob J) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t bar_b[2];    // table chunk landed (bulk copy)
  __shared__ __align__(8) uint64_t bar_m[2];    // MMAs of the stage done (tcgen05.commit)
  __shared__ uint32_t tmem_base;
  __shared__ int fail, skip;
  __shared__ unsigned int rmax[kRows];          // |x| maxima of the data rows (FP32 bits)
  __shared__ float rscale[kRows];               // 2^(7 - e_r)
  __shared__ float rout[kRows];                 // 2^(e_r - 14)
  __shared__ float ssig[2 * 512];               // table row scales sigma[table][o]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base)), "r"(kTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bar_b[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bar_m[s])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
    fail = 0;
  }
  for (int i = tid; i < J.ntab * J.nopad; i += kThreads) ssig[i] = __ldg(J.sigma + i);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  long long g = 0;   // chunks issued by this CTA (stage g & 1)
  // data slices: thread -> (column m, k-group kg); rows m (real) and m + 64 (imaginary)
  // thread -> (column m, k-group kg of 8, half kh of it); a half-warp covers
  // the 8 rows x 16 bytes of one core matrix, so its stores do not conflict
  const int kh = tid & 1, m = (tid >> 1) & 63, kg = tid >> 7;
  const int i_th = kg * 8 + kh * kVals;            // first contraction index in the chunk
  const int quad = warp & 3, q4 = warp >> 2;       // TMEM lane group, column quarter
  const int row = quad * 32 + lane;                 // TMEM lane = data row
  const int mc = row & 63, part = row >> 6;         // tile column, real / imaginary part
  bool stop = false;
  // work items: tiles, or (tile, pass) pairs when tiles are too few to fill the GPU
  const long long nitems = J.ntiles * (J.split ? J.npass : 1);
  for (long long it = blockIdx.x; it < nitems && !stop; it += gridDim.x) {
    const long long t = J.split ? it / J.npass : it;
    const int pass0 = J.split ? (int)(it % J.npass) : 0;
    const int pass1 = J.split ? pass0 + 1 : J.npass;
    const int cb = (int)(t % J.ntcol);
    const long long bf = t / J.ntcol;
    const int f = (int)(bf % J.nsrc), b = (int)(bf / J.nsrc);
    // one read of the member's status for the whole CTA (the diagnostics
    // of the previous step may set it while this kernel runs)
    if (tid == 0) skip = (J.status && J.status[b]) ? 1 : 0;
    if (tid < kRows) rmax[tid] = 0u;
    __syncthreads();
    const int sk = skip;
    __syncthreads();
    if (sk) continue;
    bool any = false;
    for (int pass = pass0; pass < pass1; ++pass)
      for (int u = J.p_u0[pass]; u < J.p_u0[pass] + J.p_nu[pass]; ++u) any |= (J.dst[J.u_tab[u]][f] >= 0);
    if (!any) continue;
    const int col0 = cb * kCols;
    const int ncv = min(kCols, J.ncol - col0);
    const char* inb = static_cast<const char*>(J.in) + (b * J.in_ms + f * J.in_fs) * (F64 ? 16 : 8);
    // row exponents: 2^e_r > max |x_r| >= 2^(e_r - 1), from the largest
    // magnitude's bit pattern (two chunks in flight)
    {
      float mre = 0.f, mim = 0.f;
      for (int kc = 0; kc < J.nchunk; kc += 2) {
        Raw<F64> r0, r1;
        load_raw<F64>(J, inb, col0, ncv, kc * kChunk + i_th, m, r0);
        load_raw<F64>(J, inb, col0, ncv, (kc + 1) * kChunk + i_th, m, r1);
        if constexpr (F64) {
          unsigned long long ar = 0ull, ai = 0ull;
          const unsigned long long mask = 0x7FFFFFFFFFFFFFFFull;
#pragma unroll
          for (int e = 0; e < kVals; ++e) {
            ar = max(ar, (unsigned long long)__double_as_longlong(r0.v[e].x) & mask);
            ai = max(ai, (unsigned long long)__double_as_longlong(r0.v[e].y) & mask);
            ar = max(ar, (unsigned long long)__double_as_longlong(r1.v[e].x) & mask);
            ai = max(ai, (unsigned long long)__double_as_longlong(r1.v[e].y) & mask);
          }
          mre = fmaxf(mre, f64_to_f32_trunc(__longlong_as_double((long long)ar)));
          mim = fmaxf(mim, f64_to_f32_trunc(__longlong_as_double((long long)ai)));
        } else {
#pragma unroll
          for (int e = 0; e < kVals; ++e) {
            mre = fmaxf(mre, fmaxf(fabsf(r0.v[e].x), fabsf(r1.v[e].x)));
            mim = fmaxf(mim, fmaxf(fabsf(r0.v[e].y), fabsf(r1.v[e].y)));
          }
        }
      }
      atomicMax(&rmax[m], __float_as_uint(mre));
      atomicMax(&rmax[m + 64], __float_as_uint(mim));
      __syncthreads();
      if (tid < kRows) {
        int e = 0;
        frexpf(__uint_as_float(rmax[tid]), &e);
        // rows below 2^-100 (far under any value of the fields here) are
        // taken as zero, so that the scale stays finite
        rscale[tid] = (e < -100) ? 0.f : ldexpf(1.f, 7 - e);
        rout[tid] = ldexpf(1.f, max(e, -100) - 14);
      }
      __syncthreads();
    }
    for (int pass = pass0; pass < pass1 && !stop; ++pass) {
      const int ua = J.p_u0[pass], ub = ua + J.p_nu[pass];
      bool anyp = false;
      for (int u = ua; u < ub; ++u) anyp |= (J.dst[J.u_tab[u]][f] >= 0);
      if (!anyp) continue;
      Raw<F64> cur;
      load_raw<F64>(J, inb, col0, ncv, i_th, m, cur);
      for (int kc = 0; kc < J.nchunk; ++kc, ++g) {
        const int s = (int)(g & 1);
        unsigned char* sA = sm + s * J.stage_bytes;
        unsigned char* sB = sA + kNPA * kPieceA;
        // the MMAs that last read this stage (chunk g - 2) must be done
        if (g >= 2 && !mbar_wait(&bar_m[s], (uint32_t)(((g - 2) >> 1) & 1))) atomicExch(&fail, 1);
        if (tid == 0 && !fail) {
          uint32_t bytes = 0;
          for (int u = ua; u < ub; ++u)
            if (J.dst[J.u_tab[u]][f] >= 0) bytes += (uint32_t)(kNPB * J.u_w[u] * 64);
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                       :: "r"(smem_u32(&bar_b[s])), "r"(bytes) : "memory");
          uint32_t boff = 0;
          for (int u = ua; u < ub; ++u) {
            const uint32_t nb = (uint32_t)(kNPB * J.u_w[u] * 64);
            if (J.dst[J.u_tab[u]][f] >= 0) {
              const unsigned char* src = J.W + J.u_goff[u] + (long long)kc * nb;
              asm volatile(
                  "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                  :: "r"(smem_u32(sB + boff)), "l"(src), "r"(nb), "r"(smem_u32(&bar_b[s])) : "memory");
            }
            boff += nb;
          }
        }
        {
          // this chunk's values, then the next chunk's loads go out before
          // this chunk is sliced, stored and multiplied
          float re[kVals], im[kVals];
          raw_values<F64>(cur, re, im);
          if (kc + 1 < J.nchunk) load_raw<F64>(J, inb, col0, ncv, (kc + 1) * kChunk + i_th, m, cur);
#pragma unroll
          for (int pt = 0; pt < 2; ++pt) {
            const int r = m + 64 * pt;
            const float sc = rscale[r];
            const float* x = pt ? im : re;
            uint32_t w[kNPA][kVals / 2];
#pragma unroll
            for (int e = 0; e < kVals; e += 2) {
              float a[kNPA], c[kNPA];
              slice4(x[e], sc, a);
              slice4(x[e + 1], sc, c);
#pragma unroll
              for (int pc = 0; pc < kNPA; ++pc) w[pc][e >> 1] = pack_bf16x2(a[pc], c[pc]);
            }
            const int off = (r >> 3) * kSBO + kg * kLBO + (r & 7) * 16 + kh * 8;
#pragma unroll
            for (int pc = 0; pc < kNPA; ++pc)
              *reinterpret_cast<uint2*>(sA + pc * kPieceA + off) = make_uint2(w[pc][0], w[pc][1]);
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        stop = fail != 0;
        if (stop) break;
        if (tid == 0) {
          if (!mbar_wait(&bar_b[s], (uint32_t)((g >> 1) & 1))) {
            atomicExch(&fail, 1);
          } else {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int nks = min(2, J.nkstep - 2 * kc);
            const uint32_t a_base = smem_u32(sA);
            uint32_t boff = 0, toff = 0;
            for (int u = ua; u < ub; ++u) {
              const int nw = J.u_w[u];
              const uint32_t piece_b = (uint32_t)nw * 64;
              if (J.dst[J.u_tab[u]][f] >= 0) {
                const uint32_t b_base = smem_u32(sB) + boff;
                const uint32_t idesc = umma_idesc(nw);
                for (int ks = 0; ks < nks; ++ks) {
                  const uint32_t kofs = ks * 2 * kLBO;
                  const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
                  // A0 += X0 W0
                  mma_bf16(tmem + toff, umma_desc(a_base + kofs), umma_desc(b_base + kofs), idesc, acc);
                  // A1 += X0 W1 + X1 W0 + X0 (W2/2^8) + X1 (W1/2^8) + (X2/2^8) W0
                  //     + X0 (W3/2^16) + X1 (W2/2^16) + (X2/2^8)(W1/2^8) + (X3/2^16) W0
                  // (data slice, table slice) pairs, slices numbered as stored
                  const uint32_t t1 = tmem + toff + (uint32_t)nw;
                  const int pa[9] = {0, 1, 0, 1, 2, 0, 1, 2, 3};
                  const int pb[9] = {1, 0, 3, 2, 0, 5, 4, 2, 0};
#pragma unroll
                  for (int q = 0; q < 9; ++q)
                    mma_bf16(t1, umma_desc(a_base + pa[q] * kPieceA + kofs),
                             umma_desc(b_base + pb[q] * piece_b + kofs), idesc, q ? 1u : acc);
                }
              }
              boff += kNPB * piece_b;
              toff += 2 * (uint32_t)nw;
            }
            mma_commit(&bar_m[s]);
          }
        }
      }
      if (stop) break;
      // epilogue: wait for the pass's last MMAs
      const long long gl = g - 1;
      if (!mbar_wait(&bar_m[gl & 1], (uint32_t)((gl >> 1) & 1))) atomicExch(&fail, 1);
      asm volatile("tcgen05.fence::after_thread_sync;");
      __syncthreads();
      stop = fail != 0;
      if (stop) break;
      const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16);
      // out = (A0 + A1/2^8) sigma_o 2^(e_r - 14), both scales powers of two
      const float so = rout[row];
      if (!J.out_f64) {
        // FP32 values, output element (column, o) at column * out_cs + o * out_os
        float* ob = static_cast<float*>(J.out);
        const long long ostep = 2 * J.out_os;
        uint32_t toff = 0;
        for (int u = ua; u < ub; ++u) {
          const int nw = J.u_w[u], tb = J.u_tab[u];
          const int d = J.dst[tb][f];
          if (d >= 0) {
            const float* sig = ssig + tb * J.nopad + J.u_o0[u];
            const long long base = b * J.out_ms + d * J.out_fs + (long long)(col0 + mc) * J.out_cs;
            for (int c0 = 16 * q4; c0 < nw; c0 += 64) {
              uint32_t r0[16], r1[16];
              __syncwarp();
              tmem_ld16x2(lane_base + toff + (uint32_t)c0, lane_base + toff + (uint32_t)(nw + c0), r0, r1);
              if (mc < ncv) {
                const int o0 = J.u_o0[u] + c0;
                float* op = ob + 2 * (base + (long long)o0 * J.out_os) + part;
                const int ne = min(16, J.nout - o0);
#pragma unroll
                for (int e = 0; e < 16; ++e)
                  if (e < ne)
                    op[e * ostep] = fmaf(__uint_as_float(r1[e]), 1.f / 256.f, __uint_as_float(r0[e])) *
                                    (sig[c0 + e] * so);
              }
            }
          }
          toff += 2 * (uint32_t)nw;
        }
      } else {
        // FP64 coefficients, output element (column, o) at column * out_cs + o (out_os = 1):
        // staged per half tile (32 columns) in shared memory, rows of 2 nout + 1 doubles
        double* st = reinterpret_cast<double*>(sm);
        const int S = 2 * J.nout + 1;
        double* ob = static_cast<double*>(J.out);
        const int d = J.dst[J.u_tab[ua]][f];
        for (int hh = 0; hh < 2; ++hh) {
          // columns 32 hh .. 32 hh + 31 sit in TMEM lanes of quads hh (real) and hh + 2 (imaginary)
          if ((quad & 1) == hh) {
            const int ml = mc - 32 * hh;
            uint32_t toff = 0;
            for (int u = ua; u < ub; ++u) {
              const int nw = J.u_w[u], tb = J.u_tab[u];
              const float* sig = ssig + tb * J.nopad + J.u_o0[u];
              for (int c0 = 16 * q4; c0 < nw; c0 += 64) {
                uint32_t r0[16], r1[16];
                __syncwarp();
                tmem_ld16x2(lane_base + toff + (uint32_t)c0, lane_base + toff + (uint32_t)(nw + c0), r0, r1);
                const int o0 = J.u_o0[u] + c0;
                const int ne = min(16, J.nout - o0);
                double* sp = st + ml * S + 2 * o0 + part;
#pragma unroll
                for (int e = 0; e < 16; ++e)
                  if (e < ne)
                    sp[2 * e] = f32_to_f64_bits(fmaf(__uint_as_float(r1[e]), 1.f / 256.f,
                                                     __uint_as_float(r0[e])) * (sig[c0 + e] * so));
              }
              toff += 2 * (uint32_t)nw;
            }
          }
          __syncthreads();
          // the outputs o_lo <= o < o_hi of this pass, row by row
          const int nmh = max(0, min(32, ncv - 32 * hh));
          const int o_lo = J.u_o0[ua];
          const int o_hi = min(J.nout, J.u_o0[ub - 1] + J.u_w[ub - 1]);
          if (d >= 0 && nmh > 0 && o_hi > o_lo) {
            const long long base = b * J.out_ms + d * J.out_fs + (long long)(col0 + 32 * hh) * J.out_cs;
            // one warp per row, lanes along the row
            for (int ml = warp; ml < nmh; ml += kThreads / 32) {
              double* orow = ob + 2 * (base + (long long)ml * J.out_cs);
              const double* srow = st + ml * S;
              for (int rem = 2 * o_lo + lane; rem < 2 * o_hi; rem += 32) orow[rem] = srow[rem];
            }
          }
          __syncthreads();
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;");
    }
  }
  // drain: no MMA or bulk copy of this CTA may still be in flight at exit
  __syncthreads();
  if (fail && tid == 0) atomicExch(J.err, 1);
  if (tid == 0 && g > 0) {
    // after a failure the chunk that stopped the loop may have a copy in flight
    const long long gend = fail ? g + 1 : g;
    for (long long gg = (g >= 2 ? g - 2 : 0); gg < gend; ++gg) {
      mbar_wait(&bar_m[gg & 1], (uint32_t)((gg >> 1) & 1));
      mbar_wait(&bar_b[gg & 1], (uint32_t)((gg >> 1) & 1));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTmemCols));
}

// ------------------------------------------------------------- host side
// Units (table, output subtile of <= 256 rows, a multiple of 16), packed
// into passes whose accumulators (two per output row) fit the tensor memory.
struct Geom {
  int kin, nout, ntab;
  int nkstep, nchunk, nopad;
  int nunit, u_tab[kMaxUnits], u_o0[kMaxUnits], u_w[kMaxUnits];
  long long u_goff[kMaxUnits];
  int npass, p_u0[kMaxPass], p_nu[kMaxPass];
  long long wbytes;     // sliced tables
  int stage_bytes, smem;
};

Geom geom(int kin, int nout, int ntab, bool f64_out) {
  Geom G{};
  G.kin = kin;
  G.nout = nout;
  G.ntab = ntab;
  G.nkstep = (kin + 15) / 16;
  G.nchunk = (G.nkstep + 1) / 2;
  G.nopad = (nout + 15) / 16 * 16;
  // output subtiles: at most kMaxW rows each, multiples of 16, near-equal
  const int nsub = (G.nopad + kMaxW - 1) / kMaxW;
  int sub[kMaxUnits] = {};
  {
    int left = G.nopad / 16;
    for (int q = 0; q < nsub; ++q) {
      const int w16 = (left + (nsub - q) - 1) / (nsub - q);
      sub[q] = 16 * w16;
      left -= w16;
    }
  }
  long long goff = 0;
  for (int tb = 0; tb < ntab; ++tb) {
    int o0 = 0;
    for (int q = 0; q < nsub && G.nunit < kMaxUnits; ++q) {
      const int u = G.nunit++;
      G.u_tab[u] = tb;
      G.u_o0[u] = o0;
      G.u_w[u] = sub[q];
      G.u_goff[u] = goff;
      goff += (long long)G.nchunk * kNPB * sub[q] * 64;
      o0 += sub[q];
    }
  }
  G.wbytes = goff;
  // passes: consecutive units while their accumulators (2 w columns each)
  // fit the tensor memory and their two stages fit shared memory
  int maxb = 0;
  for (int u = 0; u < G.nunit && G.npass < kMaxPass;) {
    const int p = G.npass++;
    G.p_u0[p] = u;
    int cols = 0, bb = 0;
    while (u < G.nunit) {
      const int c2 = cols + 2 * G.u_w[u], b2 = bb + kNPB * G.u_w[u] * 64;
      if (u > G.p_u0[p] && (c2 > kTmemCols || 2 * (kNPA * kPieceA + b2) + 1024 > kSmemLimit)) break;
      cols = c2;
      bb = b2;
      ++u;
    }
    G.p_nu[p] = u - G.p_u0[p];
    maxb = std::max(maxb, bb);
  }
  G.stage_bytes = kNPA * kPieceA + maxb;
  int sm = 2 * G.stage_bytes;
  if (f64_out) sm = std::max(sm, 32 * (2 * nout + 1) * 8);
  G.smem = sm + 1024;
  return G;
}

// cos and sin of 2 pi k / n with the angle reduced in exact integers.
void cis_host(long long k, long long n, double* c, double* s) {
  k %= n;
  if (k < 0) k += n;
  const double a = 2.0 * 3.14159265358979323846 * (double)k / (double)n;
  *c = std::cos(a);
  *s = std::sin(a);
}

uint16_t bf16_bits(double v) {   // v exact in BF16 (a small integer or one over 2^8)
  const float f = (float)v;
  uint32_t b;
  std::memcpy(&b, &f, 4);
  return (uint16_t)(b >> 16);
}

// Table entry w[o][i] of one direction.
double table_entry(int M, bool inverse, int tb, int o, int i) {
  double c, s;
  if (inverse) {
    // o = j (Gauss point), i = n (Chebyshev index); theta_j = 2 pi (2j+1) / (4M)
    cis_host((long long)i * (2 * o + 1), 4LL * M, &c, &s);
    if (tb == 0) return c;
    double c1, s1;
    cis_host(2 * o + 1, 4LL * M, &c1, &s1);
    return (double)i * s / s1;
  }
  // o = k (Chebyshev index), i = j (Gauss point)
  cis_host((long long)o * (2 * i + 1), 4LL * M, &c, &s);
  return (o == 0 ? 1.0 : 2.0) / M * c;
}

// Sliced tables in the kernel's layout, [unit][chunk][slice][w rows x 32 k]
// with core matrix (rg, kg) at rg * kSBO + kg * kLBO, row r & 7 at
// 16 (r & 7) bytes, element k & 7 at 2 (k & 7); then the row scales
// sigma[table][nopad] (FP32).
void build_tables(int M, int N, bool inverse, std::vector<uint16_t>& out) {
  const int kin = inverse ? N : M, nout = inverse ? M : N, ntab = inverse ? 2 : 1;
  const Geom G = geom(kin, nout, ntab, !inverse);
  out.assign((size_t)(G.wbytes / 2) + (size_t)ntab * G.nopad * 2, 0);
  std::vector<float> sig((size_t)ntab * G.nopad, 1.0f);
  for (int u = 0; u < G.nunit; ++u) {
    const int tb = G.u_tab[u];
    for (int oo = 0; oo < G.u_w[u]; ++oo) {
      const int o = G.u_o0[u] + oo;
      if (o >= nout) continue;
      double mx = 0.0;
      for (int i = 0; i < kin; ++i) mx = std::max(mx, std::fabs(table_entry(M, inverse, tb, o, i)));
      int e = 0;
      std::frexp(mx, &e);                    // 2^e > mx >= 2^(e-1) (e = 0 for mx = 0)
      const double sg = std::ldexp(1.0, e);
      sig[(size_t)tb * G.nopad + o] = (float)sg;
      for (int i = 0; i < kin; ++i) {
        // w / sigma * 2^7 = W0 + W1/2^8 + W2/2^16 + W3/2^24 + (|rest| <= 2^-25)
        double xs = table_entry(M, inverse, tb, o, i) / sg * 128.0;
        double wq[4];
        for (int q = 0; q < 4; ++q) {
          wq[q] = std::nearbyint(xs);
          xs = (xs - wq[q]) * 256.0;
        }
        const uint16_t sl[kNPB] = {bf16_bits(wq[0]), bf16_bits(wq[1]), bf16_bits(wq[1] / 256.0),
                                   bf16_bits(wq[2] / 256.0), bf16_bits(wq[2] / 65536.0),
                                   bf16_bits(wq[3] / 65536.0)};
        const int kc = i / kChunk, k = i % kChunk;
        const long long off = G.u_goff[u] + (long long)kc * kNPB * G.u_w[u] * 64;
        const long long in_piece = (long long)(oo >> 3) * kSBO + (k >> 3) * kLBO + (oo & 7) * 16 + (k & 7) * 2;
        for (int pc = 0; pc < kNPB; ++pc)
          out[(size_t)((off + (long long)pc * G.u_w[u] * 64 + in_piece) / 2)] = sl[pc];
      }
    }
  }
  std::memcpy(out.data() + G.wbytes / 2, sig.data(), sig.size() * sizeof(float));
}

}  // namespace

bool cheb_mma_supported(int M, int N) {
  const Geom a = geom(N, M, 2, false), b = geom(M, N, 1, true);
  auto covered = [](const Geom& G) {
    int o = 0;
    for (int u = 0; u < G.nunit; ++u) o += (G.u_tab[u] == 0) ? G.u_w[u] : 0;
    int nu = 0;
    for (int p = 0; p < G.npass; ++p) nu += G.p_nu[p];
    return o == G.nopad && nu == G.nunit && G.nunit == G.ntab * (G.nunit / G.ntab);
  };
  // 2^14 kin < 2^24 keeps the leading accumulator exact
  // the row scales of all tables sit in shared memory (1024 floats)
  return a.kin <= 1000 && b.kin <= 1000 && covered(a) && covered(b) && a.smem <= kSmemLimit &&
         b.smem <= kSmemLimit && a.ntab * a.nopad <= 1024 && b.ntab * b.nopad <= 1024;
}

size_t cheb_mma_table_bytes(int M, int N, int inverse) {
  const Geom G = inverse ? geom(N, M, 2, false) : geom(M, N, 1, true);
  return (size_t)G.wbytes + (size_t)G.ntab * G.nopad * sizeof(float);
}

void cheb_mma_tables(int M, int N, int inverse, std::vector<uint16_t>& out) {
  build_tables(M, N, inverse != 0, out);
}

template <bool F64>
cudaError_t optin_mma(int optin_bytes) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, k_cheb_mma<F64>);
  if (e) return e;
  return cudaFuncSetAttribute(k_cheb_mma<F64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              std::min(kSmemLimit, optin_bytes - (int)a.sharedSizeBytes));
}

cudaError_t set_cheb_mma_attributes(int optin_bytes) {
  cudaError_t e = optin_mma<true>(optin_bytes);
  if (!e) e = optin_mma<false>(optin_bytes);
  return e;
}

// One Chebyshev pass of a mixed group on the tensor cores (see the file
// comment).  Inverse: the nf state fields (FP64, [member][field][column][n])
// to values and y-derivatives on the padded grid (FP32,
// [member][field][j][column]); forward: nf product fields (FP32, same value
// layout) to truncated coefficients (FP64, [member][field][column][n]).
cudaError_t launch_cheb_mma(const GroupDev& g, bool inverse, cudaStream_t st, int sms) {
  const bool d3 = g.nz > 1;
  const int M = g.M, N = g.N, KZ = g.KZ;
  const int nf = d3 ? 9 : 5;
  const long long NK = (long long)N * KZ, yplane = (long long)M * KZ;
  const Geom G = inverse ? geom(N, M, 2, false) : geom(M, N, 1, true);
  MmaJob J{};
  if (inverse) {
    J.in = g.X;
    J.in_f64 = 1;
    J.in_ms = nf * NK; J.in_fs = NK; J.in_cs = N; J.in_is = 1;
    J.out = d3 ? (void*)g.Y3f : (void*)g.Ypf;
    J.out_f64 = 0;
    const int nyf = d3 ? 17 : 9;
    J.out_ms = nyf * yplane; J.out_fs = yplane; J.out_cs = 1; J.out_os = KZ;
    if (d3) {
      const int d1[9] = {9, -1, 10, 11, 12, 13, 14, 15, 16};
      for (int f = 0; f < 9; ++f) { J.dst[0][f] = f; J.dst[1][f] = d1[f]; }
    } else {
      // Yp fields: 0 u, 1 v, 2 du/dy, 3 cxx, 4 cxy, 5 cyy, 6-8 d/dy of cxx, cxy, cyy
      const int d0[5] = {0, 1, 3, 4, 5}, d1[5] = {2, -1, 6, 7, 8};
      for (int f = 0; f < 5; ++f) { J.dst[0][f] = d0[f]; J.dst[1][f] = d1[f]; }
    }
    J.W = reinterpret_cast<const unsigned char*>(g.Wyi);
  } else {
    J.in = d3 ? (const void*)g.V3f : (const void*)g.Zpf;
    J.in_f64 = 0;
    J.in_ms = nf * yplane; J.in_fs = yplane; J.in_cs = 1; J.in_is = KZ;
    J.out = g.NR;
    J.out_f64 = 1;
    J.out_ms = nf * NK; J.out_fs = NK; J.out_cs = N; J.out_os = 1;
    for (int f = 0; f < nf; ++f) { J.dst[0][f] = f; J.dst[1][f] = -1; }
    J.W = reinterpret_cast<const unsigned char*>(g.Wyf);
  }
  J.sigma = reinterpret_cast<const float*>(J.W + G.wbytes);
  J.ncol = KZ;
  J.kin = G.kin;
  J.nout = G.nout;
  J.nkstep = G.nkstep;
  J.nchunk = G.nchunk;
  J.nopad = G.nopad;
  J.nunit = G.nunit;
  for (int u = 0; u < G.nunit; ++u) {
    J.u_tab[u] = G.u_tab[u];
    J.u_o0[u] = G.u_o0[u];
    J.u_w[u] = G.u_w[u];
    J.u_goff[u] = G.u_goff[u];
  }
  J.npass = G.npass;
  for (int p = 0; p < G.npass; ++p) { J.p_u0[p] = G.p_u0[p]; J.p_nu[p] = G.p_nu[p]; }
  J.nsrc = nf;
  J.ntab = G.ntab;
  J.ntcol = (KZ + kCols - 1) / kCols;
  J.ntiles = (long long)g.nb * nf * J.ntcol;
  J.status = g.status;
  J.err = g.mma_err;
  J.stage_bytes = G.stage_bytes;
  // tiles too few for two waves over the GPU: one work item per (tile, pass)
  J.split = (J.npass > 1 && J.ntiles < 2LL * std::max(1, sms)) ? 1 : 0;
  const long long items = J.ntiles * (J.split ? J.npass : 1);
  const long long grid = std::min<long long>(items, (long long)std::max(1, sms));
  if (inverse) k_cheb_mma<true><<<(unsigned)grid, kThreads, G.smem, st>>>(J);
  else k_cheb_mma<false><<<(unsigned)grid, kThreads, G.smem, st>>>(J);
  return cudaGetLastError();
}

}  // namespace ptt
