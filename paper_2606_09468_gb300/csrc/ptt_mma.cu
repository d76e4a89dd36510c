// Chebyshev transforms of the mixed-precision step as dense contractions on
// the tensor cores (tcgen05, sm_103a), with split-BF16 compensated products
// accumulated in FP32.
//
// Along y the method (Sec. 2: Fourier-Chebyshev pseudo-spectral) maps the
// Chebyshev coefficients a_n (n < N) of every Fourier column to values on the
// padded grid of M Gauss points y_j = cos(theta_j), theta_j = pi (2j+1)/(2M):
//   inverse  f_j  = sum_n T_n(y_j) a_n,          f'_j = sum_n T_n'(y_j) a_n,
//            T_n(y_j) = cos(n theta_j),  T_n'(y_j) = n sin(n theta_j) / sin(theta_j)
//   forward  a_k  = s_k sum_j cos(k theta_j) f_j  (k < N; s_0 = 1/M, s_k = 2/M),
// i.e. one matrix W (M x N, or N x M) applied to every column.  With the
// columns' real and imaginary parts as the rows of the data operand D
// (128 per tile), each transform is OUT[128 x nout] = D[128 x kin] W^T.
//
// Precision: every FP32 value x (FP64 inputs are first truncated to FP32 by
// integer operations on their bits) is split exactly into three BF16 pieces
// x = x0 + x1 + x2 (x0 = x with the low 16 bits cleared, x1 the same of
// x - x0, x2 = x - x0 - x1, which has at most 8 significant bits).  The
// tables are split the same way on the host.  Of the nine products the six
// with i + j <= 2 are accumulated in FP32 in tensor memory: the dropped ones
// are below 2^-24 of |x||w|, so the contraction keeps FP32 accuracy.  Each
// column is split relative to its own values, so a fluctuation column keeps
// its own relative accuracy however large the mean-mode column (the base
// state, whose stretch components reach 10^4) is.
//
// Kernel structure (k_cheb_mma): persistent, one CTA of 256 threads per SM,
// each CTA walking tiles (member, field, 64 Fourier columns).  Per tile the
// contraction runs in chunks of 32 along kin through a two-stage ring in
// shared memory: all threads load the chunk's data (coalesced along the
// contiguous direction of the input), split it and store the three pieces
// in the canonical K-major layout (core matrices of 8 rows x 16 bytes), while
// thread 0 brings the chunk of the pre-split table with a bulk copy
// (cp.async.bulk, completion on an mbarrier) and issues the tcgen05.mma
// instructions of the previous chunk; tcgen05.commit on a per-stage mbarrier
// frees the stage.  The epilogue reads the FP32 accumulators with
// tcgen05.ld: inverse outputs ([j][column], FP32) go straight to global
// memory, forward outputs ([column][k], FP64) through shared memory so that
// the writes are contiguous.  Every wait is bounded; a wait that runs out
// sets *err and the CTA stops after a bounded wait for its own copies.
#include <cstdint>
#include <cstring>
#include <vector>

#include "ptt_internal.h"

namespace ptt {

namespace {

constexpr int kThreads = 256;
constexpr int kRows = 128;                 // data rows per tile (64 complex columns)
constexpr int kCols = 64;                  // complex columns per tile
constexpr int kChunk = 32;                 // contraction elements per chunk (2 MMA k-steps)
constexpr int kPieceA = kRows * kChunk * 2;  // bytes of one BF16 piece of the data chunk
constexpr int kLBO = 128;                  // core-matrix stride along K (bytes)
constexpr int kSBO = 512;                  // core-matrix stride along rows (4 core matrices of K)
constexpr long long kSpin = 1LL << 26;     // iteration limit of every wait
constexpr int kSmemLimit = 227 * 1024 - 4096;  // dynamic shared memory of one CTA

struct MmaJob {
  const void* in;
  void* out;
  long long in_ms, in_fs, in_cs, in_is;    // complex-element strides: member, field, column, index
  long long out_ms, out_fs, out_cs, out_os;
  int in_f64, out_f64;
  int col_fast;        // 1: input contiguous along columns (forward), 0: along the index (inverse)
  int ncol, kin, nout;
  int nkstep, nchunk;  // 16-wide k-steps, 32-wide chunks
  int nopad;           // nout rounded up to 16
  int nsub, sub_w[2];  // MMA N-subtiles of a table (widths, sum = nopad)
  int ntab, tpp, npass;
  int nsrc;
  int dst[2][9];       // output field per (table, source field); -1: none
  const unsigned char* W;  // tables [table][chunk][piece][nopad x 32 canonical], BF16
  long long wtab;      // bytes per table
  int ntcol;           // column tiles per (member, field)
  long long ntiles;
  const int* status;
  int* err;
  int stage_bytes, a_bytes;
  int tmem_cols;
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

// FP32 bits of an FP64 value, mantissa truncated, by integer operations
// (the FP64 pipe is slow on this part): zero and values below the FP32
// normal range give a signed zero, values beyond it infinity, NaN stays NaN.
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

// Exact three-way BF16 split of x (bit patterns, high halves of FP32 values).
__device__ __forceinline__ void split3(float x, uint32_t& p0, uint32_t& p1, uint32_t& p2) {
  const uint32_t b0 = __float_as_uint(x) & 0xFFFF0000u;
  const float r1 = x - __uint_as_float(b0);
  const uint32_t b1 = __float_as_uint(r1) & 0xFFFF0000u;
  const float r2 = r1 - __uint_as_float(b1);
  p0 = b0 >> 16;
  p1 = b1 >> 16;
  p2 = __float_as_uint(r2) >> 16;   // r2 has at most 8 significant bits: exact
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Data chunk kc of tile column col0: 8 consecutive contraction indices of
// column m (rows m and m + 64 of the data operand), split into the three
// BF16 pieces and stored in the canonical layout of stage sA.
__device__ __forceinline__ void load_chunk(const MmaJob& J, const char* inb, int col0, int ncv, int kc,
                                           int m, int kg, unsigned char* sA) {
  float re[8], im[8];
  const int i0 = kc * kChunk + kg * 8;
  const bool colok = m < ncv;
  if (J.in_f64) {
    const double2* p = reinterpret_cast<const double2*>(inb) + (long long)(col0 + m) * J.in_cs;
    double2 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int i = i0 + e;
      v[e] = (colok && i < J.kin) ? __ldg(p + (long long)i * J.in_is) : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) { re[e] = f64_to_f32_trunc(v[e].x); im[e] = f64_to_f32_trunc(v[e].y); }
  } else {
    const float2* p = reinterpret_cast<const float2*>(inb) + (long long)(col0 + m) * J.in_cs;
    float2 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int i = i0 + e;
      v[e] = (colok && i < J.kin) ? __ldg(p + (long long)i * J.in_is) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) { re[e] = v[e].x; im[e] = v[e].y; }
  }
#pragma unroll
  for (int part = 0; part < 2; ++part) {
    const float* x = part ? im : re;
    uint32_t w[3][4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      uint32_t a0, a1, a2, b0, b1, b2;
      split3(x[e], a0, a1, a2);
      split3(x[e + 1], b0, b1, b2);
      w[0][e >> 1] = a0 | (b0 << 16);
      w[1][e >> 1] = a1 | (b1 << 16);
      w[2][e >> 1] = a2 | (b2 << 16);
    }
    const int r = m + 64 * part;
    const int off = (r >> 3) * kSBO + kg * kLBO + (r & 7) * 16;
#pragma unroll
    for (int pc = 0; pc < 3; ++pc)
      *reinterpret_cast<uint4*>(sA + pc * kPieceA + off) = make_uint4(w[pc][0], w[pc][1], w[pc][2], w[pc][3]);
  }
}

__global__ void __launch_bounds__(kThreads, 1) k_cheb_mma(MmaJob J) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t bar_b[2];    // table chunk landed (bulk copy)
  __shared__ __align__(8) uint64_t bar_m[2];    // MMAs of the stage done (tcgen05.commit)
  __shared__ uint32_t tmem_base;
  __shared__ int fail, skip;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base)), "r"(J.tmem_cols) : "memory");
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
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t bchunk = (uint32_t)(J.wtab / J.nchunk);   // bytes of one table chunk
  long long g = 0;   // chunks issued by this CTA (stage g & 1)
  // data pieces: thread -> (column m, k-group kg); rows m (real) and m + 64 (imaginary)
  const int m = tid & 63, kg = tid >> 6;
  const int quad = warp & 3, half = warp >> 2;
  const int row = quad * 32 + lane;                 // TMEM lane = data row
  const int mc = row & 63, part = row >> 6;         // tile column, real / imaginary part
  bool stop = false;
  for (long long t = blockIdx.x; t < J.ntiles && !stop; t += gridDim.x) {
    const int cb = (int)(t % J.ntcol);
    const long long bf = t / J.ntcol;
    const int f = (int)(bf % J.nsrc), b = (int)(bf / J.nsrc);
    // one read of the member's status for the whole CTA (the diagnostics
    // of the previous step may set it while this kernel runs)
    if (tid == 0) skip = (J.status && J.status[b]) ? 1 : 0;
    __syncthreads();
    const int sk = skip;
    __syncthreads();
    if (sk) continue;
    const int col0 = cb * kCols;
    const int ncv = min(kCols, J.ncol - col0);
    const char* inb = static_cast<const char*>(J.in) + (b * J.in_ms + f * J.in_fs) * (J.in_f64 ? 16 : 8);
    for (int pass = 0; pass < J.npass && !stop; ++pass) {
      const int t0 = pass * J.tpp, t1 = min(J.ntab, t0 + J.tpp);
      bool any = false;
      for (int tb = t0; tb < t1; ++tb) any |= (J.dst[tb][f] >= 0);
      if (!any) continue;
      for (int kc = 0; kc < J.nchunk; ++kc, ++g) {
        const int s = (int)(g & 1);
        unsigned char* sA = sm + s * J.stage_bytes;
        unsigned char* sB = sA + J.a_bytes;
        // the MMAs that last read this stage (chunk g - 2) must be done
        if (g >= 2 && !mbar_wait(&bar_m[s], (uint32_t)(((g - 2) >> 1) & 1))) atomicExch(&fail, 1);
        if (tid == 0 && !fail) {
          uint32_t bytes = 0;
          for (int tb = t0; tb < t1; ++tb)
            if (J.dst[tb][f] >= 0) bytes += bchunk;
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                       :: "r"(smem_u32(&bar_b[s])), "r"(bytes) : "memory");
          for (int tb = t0; tb < t1; ++tb) {
            if (J.dst[tb][f] < 0) continue;
            const unsigned char* src = J.W + tb * J.wtab + (long long)kc * bchunk;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                :: "r"(smem_u32(sB + (tb - t0) * bchunk)), "l"(src), "r"(bchunk), "r"(smem_u32(&bar_b[s]))
                : "memory");
          }
        }
        load_chunk(J, inb, col0, ncv, kc, m, kg, sA);
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
            const uint32_t piece_b = (uint32_t)J.nopad * 64;
            for (int tb = t0; tb < t1; ++tb) {
              if (J.dst[tb][f] < 0) continue;
              const uint32_t b_base = smem_u32(sB) + (uint32_t)(tb - t0) * bchunk;
              int u0 = 0;
              for (int u = 0; u < J.nsub; ++u) {
                const int nw = J.sub_w[u];
                const uint32_t idesc = umma_idesc(nw);
                const uint32_t dcol = tmem + (uint32_t)((tb - t0) * J.nopad + u0);
                for (int ks = 0; ks < nks; ++ks) {
                  // products x_i w_j with i + j <= 2
#pragma unroll
                  for (int q = 0; q < 6; ++q) {
                    const int pa = (q == 2 || q == 4) ? 1 : (q == 5 ? 2 : 0);
                    const int pb = (q == 1 || q == 4) ? 1 : (q == 3 ? 2 : 0);
                    const uint64_t ad = umma_desc(a_base + pa * kPieceA + ks * 2 * kLBO);
                    const uint64_t bd = umma_desc(b_base + pb * piece_b + (u0 >> 3) * kSBO + ks * 2 * kLBO);
                    const uint32_t acc = (kc > 0 || ks > 0 || q > 0) ? 1u : 0u;
                    mma_bf16(dcol, ad, bd, idesc, acc);
                  }
                }
                u0 += nw;
              }
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
      const int ncols = (t1 - t0) * J.nopad;
      if (!J.out_f64) {
        // FP32 values, output element (column, o) at column * out_cs + o * out_os
        float* ob = static_cast<float*>(J.out);
        for (int c0 = 16 * half; c0 < ncols; c0 += 32) {
          uint32_t r[16];
          __syncwarp();
          tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0, r);
          const int tb = t0 + c0 / J.nopad;
          const int d = J.dst[tb][f];
          if (d >= 0 && mc < ncv) {
            const long long base = b * J.out_ms + d * J.out_fs + (long long)(col0 + mc) * J.out_cs;
            const int oc = c0 % J.nopad;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const int o = oc + e;
              if (o < J.nout) ob[2 * (base + (long long)o * J.out_os) + part] = __uint_as_float(r[e]);
            }
          }
        }
      } else {
        // FP64 coefficients, output element (column, o) at column * out_cs + o (out_os = 1):
        // staged per half tile (32 columns) in shared memory, rows of 2 nout + 1 doubles
        double* st = reinterpret_cast<double*>(sm);
        const int S = 2 * J.nout + 1;
        const int d = J.dst[t0][f];
        double* ob = static_cast<double*>(J.out);
        for (int hh = 0; hh < 2; ++hh) {
          // columns 32 hh .. 32 hh + 31 sit in TMEM lanes of quads hh (real) and hh + 2 (imaginary)
          if ((quad & 1) == hh) {
            const int ml = mc - 32 * hh;
            for (int c0 = 16 * half; c0 < J.nopad; c0 += 32) {
              uint32_t r[16];
              __syncwarp();
              tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0, r);
#pragma unroll
              for (int e = 0; e < 16; ++e) {
                const int o = c0 + e;
                if (o < J.nout) st[ml * S + 2 * o + part] = (double)__uint_as_float(r[e]);
              }
            }
          }
          __syncthreads();
          const int nmh = max(0, min(32, ncv - 32 * hh));
          if (d >= 0 && nmh > 0) {
            const long long base = b * J.out_ms + d * J.out_fs + (long long)(col0 + 32 * hh) * J.out_cs;
            const int rowd = 2 * J.nout;
            const int tot = nmh * rowd;
            for (int q = tid; q < tot; q += kThreads) {
              const int ml = q / rowd, rem = q - ml * rowd;
              ob[2 * (base + (long long)ml * J.out_cs) + rem] = st[ml * S + rem];
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(J.tmem_cols));
}

// ------------------------------------------------------------- host side
struct Geom {
  int kin, nout, ntab;
  int nkstep, nchunk, nopad, nsub, sub_w[2], tpp, npass, tmem_cols;
  long long wtab;       // bytes per table
  int a_bytes, stage_bytes, smem;
};

Geom geom(int kin, int nout, int ntab, bool f64_out) {
  Geom G{};
  G.kin = kin;
  G.nout = nout;
  G.ntab = ntab;
  G.nkstep = (kin + 15) / 16;
  G.nchunk = (G.nkstep + 1) / 2;
  G.nopad = (nout + 15) / 16 * 16;
  if (G.nopad <= 256) {
    G.nsub = 1;
    G.sub_w[0] = G.nopad;
    G.sub_w[1] = 0;
  } else {
    G.nsub = 2;
    G.sub_w[0] = (G.nopad / 2 + 15) / 16 * 16;
    G.sub_w[1] = G.nopad - G.sub_w[0];
  }
  G.wtab = (long long)G.nchunk * 3 * G.nopad * 64;
  G.a_bytes = 3 * kPieceA;
  // all tables in one pass when their accumulators fit the 512 tensor-memory
  // columns and their two stages fit shared memory, else one table per pass
  for (int tpp = ntab; tpp >= 1; --tpp) {
    G.tpp = tpp;
    G.stage_bytes = G.a_bytes + G.tpp * 3 * G.nopad * 64;
    int sm = 2 * G.stage_bytes;
    if (f64_out) sm = std::max(sm, 32 * (2 * nout + 1) * 8);
    G.smem = sm + 1024;
    if (tpp * G.nopad <= 512 && G.smem <= kSmemLimit) break;
  }
  G.npass = (ntab + G.tpp - 1) / G.tpp;
  int tc = 32;
  while (tc < G.tpp * G.nopad) tc *= 2;
  G.tmem_cols = tc;
  return G;
}

// Exact three-way BF16 split of the FP32 rounding of v (host twin of split3).
void split3_host(double v, uint16_t* p) {
  const float x = (float)v;
  uint32_t bx;
  std::memcpy(&bx, &x, 4);
  const uint32_t b0 = bx & 0xFFFF0000u;
  float f0;
  std::memcpy(&f0, &b0, 4);
  const float r1 = x - f0;
  uint32_t br1;
  std::memcpy(&br1, &r1, 4);
  const uint32_t b1 = br1 & 0xFFFF0000u;
  float f1;
  std::memcpy(&f1, &b1, 4);
  const float r2 = r1 - f1;
  uint32_t br2;
  std::memcpy(&br2, &r2, 4);
  p[0] = (uint16_t)(b0 >> 16);
  p[1] = (uint16_t)(b1 >> 16);
  p[2] = (uint16_t)(br2 >> 16);
}

// cos and sin of 2 pi k / n with the angle reduced in exact integers.
void cis_host(long long k, long long n, double* c, double* s) {
  k %= n;
  if (k < 0) k += n;
  const double a = 2.0 * 3.14159265358979323846 * (double)k / (double)n;
  *c = std::cos(a);
  *s = std::sin(a);
}

// Tables of one direction in the kernel's layout: [table][chunk][piece]
// [nopad rows x 32 k], core matrix (rg, kg) at rg * kSBO + kg * kLBO, row
// r & 7 at 16 (r & 7) bytes, element k & 7 at 2 (k & 7).
void build_tables(int M, int N, bool inverse, std::vector<uint16_t>& out, Geom& G) {
  const int kin = inverse ? N : M, nout = inverse ? M : N, ntab = inverse ? 2 : 1;
  G = geom(kin, nout, ntab, !inverse);
  out.assign((size_t)(G.wtab / 2) * ntab, 0);
  for (int tb = 0; tb < ntab; ++tb)
    for (int o = 0; o < nout; ++o)
      for (int i = 0; i < kin; ++i) {
        double w;
        if (inverse) {
          // o = j (Gauss point), i = n (Chebyshev index); theta_j = 2 pi (2j+1) / (4M)
          double c, s;
          cis_host((long long)i * (2 * o + 1), 4LL * M, &c, &s);
          if (tb == 0) {
            w = c;
          } else {
            double c1, s1;
            cis_host(2 * o + 1, 4LL * M, &c1, &s1);
            w = (double)i * s / s1;
          }
        } else {
          // o = k (Chebyshev index), i = j (Gauss point)
          double c, s;
          cis_host((long long)o * (2 * i + 1), 4LL * M, &c, &s);
          w = (o == 0 ? 1.0 : 2.0) / M * c;
        }
        uint16_t p[3];
        split3_host(w, p);
        const int kc = i / kChunk, k = i % kChunk;
        const long long off = (long long)tb * G.wtab + (long long)kc * 3 * G.nopad * 64;
        const long long in_piece = (long long)(o >> 3) * kSBO + (k >> 3) * kLBO + (o & 7) * 16 + (k & 7) * 2;
        for (int pc = 0; pc < 3; ++pc)
          out[(size_t)((off + (long long)pc * G.nopad * 64 + in_piece) / 2)] = p[pc];
      }
}

}  // namespace

bool cheb_mma_supported(int M, int N) {
  // outputs of one table within tensor memory (512 FP32 columns) and the
  // shared-memory plan within the 227 KB of one CTA
  const Geom a = geom(N, M, 2, false), b = geom(M, N, 1, true);
  return a.nopad <= 512 && b.nopad <= 512 && a.smem <= kSmemLimit && b.smem <= kSmemLimit;
}

size_t cheb_mma_table_bytes(int M, int N, int inverse) {
  const Geom G = inverse ? geom(N, M, 2, false) : geom(M, N, 1, true);
  return (size_t)G.wtab * G.ntab;
}

void cheb_mma_tables(int M, int N, int inverse, std::vector<uint16_t>& out) {
  Geom G;
  build_tables(M, N, inverse != 0, out, G);
}

size_t cheb_mma_smem(int M, int N) {
  const Geom a = geom(N, M, 2, false), b = geom(M, N, 1, true);
  return (size_t)std::max(a.smem, b.smem);
}

cudaError_t set_cheb_mma_attributes(int optin_bytes) {
  return cudaFuncSetAttribute(k_cheb_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, optin_bytes - 4096);
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
    J.col_fast = 0;
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
    J.col_fast = 1;
    for (int f = 0; f < nf; ++f) { J.dst[0][f] = f; J.dst[1][f] = -1; }
    J.W = reinterpret_cast<const unsigned char*>(g.Wyf);
  }
  J.ncol = KZ;
  J.kin = G.kin;
  J.nout = G.nout;
  J.nkstep = G.nkstep;
  J.nchunk = G.nchunk;
  J.nopad = G.nopad;
  J.nsub = G.nsub;
  J.sub_w[0] = G.sub_w[0];
  J.sub_w[1] = G.sub_w[1];
  J.ntab = G.ntab;
  J.tpp = G.tpp;
  J.npass = G.npass;
  J.nsrc = nf;
  J.wtab = G.wtab;
  J.ntcol = (KZ + kCols - 1) / kCols;
  J.ntiles = (long long)g.nb * nf * J.ntcol;
  J.status = g.status;
  J.err = g.mma_err;
  J.a_bytes = G.a_bytes;
  J.stage_bytes = G.stage_bytes;
  J.tmem_cols = G.tmem_cols;
  const long long grid = std::min<long long>(J.ntiles, (long long)std::max(1, sms));
  k_cheb_mma<<<(unsigned)grid, kThreads, G.smem, st>>>(J);
  return cudaGetLastError();
}

}  // namespace ptt
