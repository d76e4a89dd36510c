// Host side of the sPTT channel library: parameter checks, plans, operator
// tables, workspace carving, initial condition, CUDA-graph step, C ABI.
#include <algorithm>
#include <chrono>
#include <thread>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <tuple>
#include <utility>
#include <vector>

#include "ptt_internal.h"

using namespace ptt;

namespace {

constexpr double kPi = 3.14159265358979323846;

bool smooth235(long long n) {
  if (n < 1) return false;
  for (int p : {2, 3, 5})
    while (n % p == 0) n /= p;
  return n == 1;
}

// Admitted unpadded lengths: 13-smooth (one FFT pass per prime factor;
// radices 7, 11 and 13 take direct butterflies).  Padded lengths are chosen
// 5-smooth (next_smooth), where the passes are cheapest.
bool smooth13(long long n) {
  if (n < 1) return false;
  for (int p : {2, 3, 5, 7, 11, 13})
    while (n % p == 0) n /= p;
  return n == 1;
}

int next_smooth(int n) {
  while (!smooth235(n)) ++n;
  return n;
}

// cos and sin of 2 pi k / n with exact integer reduction to [0, pi/4].
void cis(long long k, long long n, double* c, double* s) {
  long long q = (4 * (k % n) + 4 * n) % (4 * n);  // angle = (pi/2) q / n, q in [0, 4n)
  double sgn_s = 1.0, sgn_c = 1.0;
  if (q > 2 * n) { q = 4 * n - q; sgn_s = -1.0; }   // (pi, 2 pi) -> (0, pi)
  if (q > n) { q = 2 * n - q; sgn_c = -1.0; }       // (pi/2, pi) -> (0, pi/2)
  bool swap = false;
  if (2 * q > n) { q = n - q; swap = true; }         // (pi/4, pi/2) -> (0, pi/4)
  const double th = 0.5 * kPi * (double)q / (double)n;
  double cc = std::cos(th), ss = std::sin(th);
  if (swap) std::swap(cc, ss);
  *c = sgn_c * cc;
  *s = sgn_s * ss;
}

struct HostPlan {
  int n = 0;
  std::vector<int> radix;
};

// three_first: the padded x and z lengths (3K or more for K kept modes).
// Their inverse lines are zero in the middle third [n/3, 2n/3), so a first
// pass of radix 3 has one zero input (8 FP64 operations per butterfly
// against 12); used where n has no factor 5.
// wide: the plans of FP32 groups may take radix-8 passes (fewer passes,
// each a shared-memory round trip; their transforms are bound by
// instruction issue, not arithmetic); the FP64 plans keep radices up to 5,
// whose tangent-form twiddles save FP64 operations, and so do the
// double-single ones (measured slower with radix 8: register pressure).
HostPlan make_plan(int n, bool three_first = false, bool wide = false) {
  HostPlan p;
  p.n = n;
  int r = n;
  if (three_first && n % 3 == 0 && n % 5 != 0) { p.radix.push_back(3); r /= 3; }
  // radix 5 first: the first pass takes no twiddles, and a twiddled radix-5
  // butterfly costs the most (44 FP64 operations against 36 untwiddled)
  // radices 13, 11, 7 (unpadded lengths only) first: their butterflies are
  // the costliest, and the first pass takes no twiddles
  for (int f : {13, 11, 7, 5})
    while (r % f == 0) { p.radix.push_back(f); r /= f; }
  if (wide)
    while (r % 8 == 0) { p.radix.push_back(8); r /= 8; }
  for (int f : {4, 2, 3})
    while (r % f == 0) { p.radix.push_back(f); r /= f; }
  return p;
}

// Quasi-tridiagonal operator tables of (alpha - beta D^2) a = R on the
// tau rows n <= N-3 with one Dirichlet-type sum row per parity.
// For parity p the unknowns a_n (n = p mod 2) satisfy, for n >= 2,
//   l_n a_{n-2} + d_n a_n + u_n a_{n+2} = r_n,
//   l_n = -alpha c_{n-2} w1_n, d_n = beta + [n <= N-3] alpha w2_n,
//   u_n = -[n <= N-5] alpha w3_n,
// w1 = 1/(4n(n-1)), w2 = 1/(2(n^2-1)), w3 = 1/(4n(n+1)), c_0 = 2, c_n = 1.
// (These rows follow from writing a_n through the coefficients of D^2 a,
// which the tau rows fix.)  Backward elimination a_n = P_n + Q_n a_{n-2};
// Q, inv = 1/(d_n + u_n Q_{n+2}) and F_n = 1 + V_{n+2} (V the coefficient of
// a_{n-2} in sum_{j >= n} a_j) do not depend on R; G = 1/(1 + V_{p+2}).
void qt_tables(int N, double alpha, double beta, const double* w1, const double* w2,
               const double* w3, int p, double* Q, double* inv, double* F, double* G,
               size_t stride) {
  const int nl = ((N - 1 - p) & ~1) + p;
  double Qn2 = 0.0, Vn2 = 0.0;
  for (int n = nl; n >= p + 2; n -= 2) {
    const double c = (n == 2) ? 2.0 : 1.0;
    const double l = -alpha * c * w1[n];
    const double d = beta + (n <= N - 3 ? alpha * w2[n] : 0.0);
    const double u = (n <= N - 5) ? -alpha * w3[n] : 0.0;
    const double iv = 1.0 / (d + u * Qn2);
    const double q = -l * iv;
    const double f = 1.0 + Vn2;
    Q[(size_t)n * stride] = q;
    inv[(size_t)n * stride] = iv;
    F[(size_t)n * stride] = f;
    Qn2 = q;
    Vn2 = f * q;
  }
  *G = 1.0 / (1.0 + Vn2);
}

// Host twin of the device solve on real data (used for the homogeneous
// solutions of the influence-matrix step).
void qt_solve_host(int N, int p, double alpha, const double* R, double* out, const double* Q,
                   const double* inv, const double* F, double G, const double* w1,
                   const double* w2, const double* w3, double g, double rsign, size_t stride) {
  const int nl = ((N - 1 - p) & ~1) + p;
  double Pn2 = 0.0, U = 0.0, Rp2 = 0.0, R0 = rsign * R[(size_t)nl * stride];
  for (int n = nl; n >= p + 2; n -= 2) {
    const double Rm2 = rsign * R[(size_t)(n - 2) * stride];
    const double c = (n == 2) ? 2.0 : 1.0;
    double r = -c * w1[n] * Rm2;
    if (n <= N - 3) r += w2[n] * R0;
    double un = 0.0;
    if (n <= N - 5) { r -= w3[n] * Rp2; un = -alpha * w3[n]; }
    const double P = (r - un * Pn2) * inv[(size_t)n * stride];
    out[(size_t)n * stride] = P;
    U += F[(size_t)n * stride] * P;
    Pn2 = P;
    Rp2 = R0;
    R0 = Rm2;
  }
  double a = (g - U) * G;
  out[(size_t)p * stride] = a;
  for (int n = p + 2; n <= nl; n += 2) {
    a = out[(size_t)n * stride] + Q[(size_t)n * stride] * a;
    out[(size_t)n * stride] = a;
  }
}

const double kSA0[4] = {1.0, 1.5, 11.0 / 6.0, 25.0 / 12.0};

// ------------------------------------------------------- initial condition
uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
// splitmix64 as a counter-based stream: output k of seed s.
double splitmix_uniform(uint64_t seed, uint64_t k) {
  const uint64_t z = mix64(seed + (k + 1) * 0x9E3779B97F4A7C15ULL);
  return 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
}

// c_xy = s of the steady laminar sPTT channel (kappa = 0): root of
// 2 beta eps s^3 + s + 2 Wi y = 0, by Newton from the Oldroyd-B value
// (monotone: the cubic is increasing, concave where the root lies).
double laminar_root(double y, double wi, double beta, double eps) {
  double s = -2.0 * wi * y;
  if (eps == 0.0 || y == 0.0) return s;
  const double a = 2.0 * beta * eps;
  for (int it = 0; it < 200; ++it) {
    const double f = a * s * s * s + s + 2.0 * wi * y;
    const double ds = f / (3.0 * a * s * s + 1.0);
    s -= ds;
    if (std::fabs(ds) <= 1e-17 * std::fabs(s)) break;
  }
  return s;
}

double laminar_F(double s, double beta, double eps) {
  const double s2 = s * s;
  return 0.5 * s2 + 0.5 * eps * (1.0 + 3.0 * beta) * s2 * s2 + 2.0 * beta * eps * eps * s2 * s2 * s2;
}

// Physical initial fields [5][ny][nx]: laminar sPTT + perturbation.
void initial_fields(const ptt_params& p, uint64_t seed, double amp, std::vector<double>& out) {
  const int nx = p.nx, ny = p.ny;
  out.assign((size_t)5 * ny * nx, 0.0);
  std::vector<double> y(ny), U(ny), cxx(ny), cxy(ny);
  const double sw = laminar_root(1.0, p.wi, p.beta, p.eps);
  const double Fw = laminar_F(sw, p.beta, p.eps);
  for (int l = 0; l < ny; ++l) {
    double c, s;
    cis(l, 2 * (ny - 1), &c, &s);  // y_l = cos(pi l/(ny-1))
    y[l] = c;
    const double r = laminar_root(c, p.wi, p.beta, p.eps);
    U[l] = -(laminar_F(r, p.beta, p.eps) - Fw) / (2.0 * p.wi * p.wi);
    cxx[l] = 1.0 + 2.0 * r * r;
    cxy[l] = r;
  }
  // perturbation: psi = (1-y^2)^2 g, g = sum_{m=1..4, n<=8} (A cos + B sin) T_n(y)
  std::vector<double> up((size_t)ny * nx, 0.0), vp((size_t)ny * nx, 0.0);
  for (int m = 1; m <= 4; ++m) {
    const double km = 2.0 * kPi * m / p.lx;
    double A[9], B[9];
    for (int n = 0; n < 9; ++n) {
      A[n] = splitmix_uniform(seed, (uint64_t)(((m - 1) * 9 + n) * 2 + 0));
      B[n] = splitmix_uniform(seed, (uint64_t)(((m - 1) * 9 + n) * 2 + 1));
    }
    for (int l = 0; l < ny; ++l) {
      const double yy = y[l];
      // T_n and T_n' = n U_{n-1} by their recurrences
      double T[9], dT[9], Uc[9];
      T[0] = 1.0; T[1] = yy;
      Uc[0] = 1.0; Uc[1] = 2.0 * yy;
      for (int n = 2; n < 9; ++n) { T[n] = 2 * yy * T[n - 1] - T[n - 2]; Uc[n] = 2 * yy * Uc[n - 1] - Uc[n - 2]; }
      dT[0] = 0.0;
      for (int n = 1; n < 9; ++n) dT[n] = n * Uc[n - 1];
      double ga = 0, gb = 0, dga = 0, dgb = 0;
      for (int n = 0; n < 9; ++n) { ga += A[n] * T[n]; gb += B[n] * T[n]; dga += A[n] * dT[n]; dgb += B[n] * dT[n]; }
      const double w = (1 - yy * yy) * (1 - yy * yy), dw = -4.0 * yy * (1 - yy * yy);
      const double pa = w * ga, pb = w * gb, dpa = dw * ga + w * dga, dpb = dw * gb + w * dgb;
      for (int j = 0; j < nx; ++j) {
        double c, s;
        cis((long long)m * j, nx, &c, &s);
        up[(size_t)l * nx + j] += dpa * c + dpb * s;
        vp[(size_t)l * nx + j] += km * (pa * s - pb * c);
      }
    }
  }
  double mx = 0.0;
  for (size_t i = 0; i < up.size(); ++i) mx = std::fmax(mx, std::sqrt(up[i] * up[i] + vp[i] * vp[i]));
  const double sc = (mx > 0.0) ? amp / mx : 0.0;
  const size_t F = (size_t)ny * nx;
  for (int l = 0; l < ny; ++l)
    for (int j = 0; j < nx; ++j) {
      const size_t i = (size_t)l * nx + j;
      out[0 * F + i] = U[l] + sc * up[i];
      out[1 * F + i] = sc * vp[i];
      out[2 * F + i] = cxx[l];
      out[3 * F + i] = cxy[l];
      out[4 * F + i] = 1.0;
    }
}

// Physical initial fields of a 3D run, [9][ny][nz][nx]: laminar sPTT +
// perturbation u' = d psi1/dy, v' = -d psi1/dx - d psi2/dz, w' = d psi2/dy,
// psi_c = (1 - y^2)^2 sum_{mx <= 4, mz <= 2, (mx, mz) != 0, n <= 8}
//         (A cos(kx x + kz z) + B sin(kx x + kz z)) T_n(y),
// A, B from the splitmix64 stream of `seed`, output
// ((((c*5 + mx)*3 + mz)*9 + n)*2 + {0, 1}); scaled to max |u'| = amp.
void initial_fields3(const ptt_params& p, uint64_t seed, double amp, std::vector<double>& out) {
  const int nx = p.nx, ny = p.ny, nz = p.nz;
  const size_t F = (size_t)ny * nz * nx;
  out.assign(9 * F, 0.0);
  std::vector<double> y(ny), U(ny), cxx(ny), cxy(ny);
  const double sw = laminar_root(1.0, p.wi, p.beta, p.eps);
  const double Fw = laminar_F(sw, p.beta, p.eps);
  for (int l = 0; l < ny; ++l) {
    double c, s;
    cis(l, 2 * (ny - 1), &c, &s);
    y[l] = c;
    const double r = laminar_root(c, p.wi, p.beta, p.eps);
    U[l] = -(laminar_F(r, p.beta, p.eps) - Fw) / (2.0 * p.wi * p.wi);
    cxx[l] = 1.0 + 2.0 * r * r;
    cxy[l] = r;
  }
  std::vector<double> up(F, 0.0), vp(F, 0.0), wp(F, 0.0);
  for (int cc = 0; cc < 2; ++cc) {
    for (int mx = 0; mx <= 4; ++mx) {
      for (int mz = 0; mz <= 2; ++mz) {
        if (mx == 0 && mz == 0) continue;
        const double kx = 2.0 * kPi * mx / p.lx, kz = 2.0 * kPi * mz / p.lz;
        double A[9], B[9];
        for (int n = 0; n < 9; ++n) {
          const uint64_t base = (uint64_t)((((cc * 5 + mx) * 3 + mz) * 9 + n) * 2);
          A[n] = splitmix_uniform(seed, base + 0);
          B[n] = splitmix_uniform(seed, base + 1);
        }
        for (int l = 0; l < ny; ++l) {
          const double yy = y[l];
          double T[9], Uc[9], dT[9];
          T[0] = 1.0; T[1] = yy; Uc[0] = 1.0; Uc[1] = 2.0 * yy;
          for (int n = 2; n < 9; ++n) { T[n] = 2 * yy * T[n - 1] - T[n - 2]; Uc[n] = 2 * yy * Uc[n - 1] - Uc[n - 2]; }
          dT[0] = 0.0;
          for (int n = 1; n < 9; ++n) dT[n] = n * Uc[n - 1];
          double ga = 0, gb = 0, dga = 0, dgb = 0;
          for (int n = 0; n < 9; ++n) { ga += A[n] * T[n]; gb += B[n] * T[n]; dga += A[n] * dT[n]; dgb += B[n] * dT[n]; }
          const double w = (1 - yy * yy) * (1 - yy * yy), dw = -4.0 * yy * (1 - yy * yy);
          const double pa = w * ga, pb = w * gb, dpa = dw * ga + w * dga, dpb = dw * gb + w * dgb;
          for (int k = 0; k < nz; ++k)
            for (int j = 0; j < nx; ++j) {
              double c, s;
              cis((long long)mx * j * nz + (long long)mz * k * nx, (long long)nx * nz, &c, &s);
              const size_t i = ((size_t)l * nz + k) * nx + j;
              const double dy = dpa * c + dpb * s;        // d psi / dy
              const double dh = -pa * s + pb * c;         // (d psi/dx)/kx = (d psi/dz)/kz
              if (cc == 0) { up[i] += dy; vp[i] -= kx * dh; }
              else { wp[i] += dy; vp[i] -= kz * dh; }
            }
        }
      }
    }
  }
  double mxv = 0.0;
  for (size_t i = 0; i < F; ++i) mxv = std::fmax(mxv, std::sqrt(up[i] * up[i] + vp[i] * vp[i] + wp[i] * wp[i]));
  const double sc = (mxv > 0.0) ? amp / mxv : 0.0;
  for (int l = 0; l < ny; ++l)
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < nx; ++j) {
        const size_t i = ((size_t)l * nz + k) * nx + j;
        out[0 * F + i] = U[l] + sc * up[i];
        out[1 * F + i] = sc * vp[i];
        out[2 * F + i] = sc * wp[i];
        out[3 * F + i] = cxx[l];
        out[4 * F + i] = cxy[l];
        out[5 * F + i] = 0.0;
        out[6 * F + i] = 1.0;
        out[7 * F + i] = 0.0;
        out[8 * F + i] = 1.0;
      }
}

// Quarter-period twiddles of the Gauss-grid (DCT-II/III) transforms on M
// points with each direction's constants folded in: fwd[k] = (s_k/2)
// exp(-i pi k/(2M)) with s_0 = 1/M, s_k = 2/M (the DCT-II normalisation of
// the coefficients), inv[k] = (1/2) exp(+i pi k/(2M)).
// A complex double as double-single parts (re.h, re.l, im.h, im.l): h the FP32
// rounding, l the FP32 rounding of the remainder (48 significant bits).
float4 ds_split(double2 v) {
  const float rh = (float)v.x, ih = (float)v.y;
  return make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
}

void quarter_tables(int M, std::vector<double2>& fwd, std::vector<double2>& inv) {
  fwd.resize(M);
  inv.resize(M);
  for (int k = 0; k < M; ++k) {
    double cc, ss;
    cis(k, 4LL * M, &cc, &ss);
    const double h = (k == 0 ? 0.5 : 1.0) / M;
    fwd[k] = make_double2(h * cc, -h * ss);
    inv[k] = make_double2(0.5 * cc, 0.5 * ss);
  }
}

// Record offsets of the tangent tables: toff[s] in records (tk), tto[s] in
// doubles (tt); *nrec and *ndbl receive the table sizes (one spare entry).
void tangent_offsets(const HostPlan& hp, int* toff, int* tto, int* nrec, int* ndbl) {
  int rec = 0, dbl = 0, Ns = 1;
  for (size_t st = 0; st < hp.radix.size(); ++st) {
    const int R = hp.radix[st];
    toff[st] = rec;
    tto[st] = dbl;
    if (st > 0 && R <= 5) {   // radices 7, 11, 13 keep plain twiddles
      rec += Ns;
      dbl += (R == 5 ? 16 : 6) * Ns;
    }
    Ns *= R;
  }
  *nrec = rec + 1;
  *ndbl = dbl + 16;
}

// Tangent-form twiddle records of an FFT plan (see FftPlan): for each pass
// s >= 1 (radix 2 to 5) and stride index jm < Ns, the forward twiddles
// w_r = exp(-2 pi i m_r / n), m_r = jm r st, written as i^k_r c_r (1 + i t_r)
// with k_r the nearest quarter turn, so that |angle of c_r + i c_r t_r| <=
// pi/4 (c_r >= 1/sqrt 2, |t_r| <= 1).
void tangent_tables(const HostPlan& hp, std::vector<double>& tt, std::vector<int>& tk) {
  const int n = hp.n;
  int toff[kMaxStages], tto[kMaxStages], nrec = 0, ndbl = 0;
  tangent_offsets(hp, toff, tto, &nrec, &ndbl);
  tt.assign((size_t)ndbl, 0.0);
  tk.assign((size_t)nrec, 0);
  double C1, S1, C2, S2;  // cos, sin of 2 pi/5 and 4 pi/5
  cis(1, 5, &C1, &S1);
  cis(2, 5, &C2, &S2);
  int Ns = 1;
  for (size_t st = 0; st < hp.radix.size(); ++st) {
    const int R = hp.radix[st];
    if (st > 0 && R <= 5) {
      const long long stride = n / ((long long)Ns * R);
      const int RS = (R == 5) ? 16 : 6;
      for (int jm = 0; jm < Ns; ++jm) {
        double c[5] = {1, 1, 1, 1, 1}, t[5] = {0, 0, 0, 0, 0};
        int kp = 0;
        for (int r = 1; r < R; ++r) {
          const long long m = ((long long)jm * r * stride) % n;
          // angle -2 pi m / n = 2 pi (-4 m) / (4 n); quarter turns k = round(-4 m / n)
          long long k = -(4 * m + n / 2) / n;             // floor((-4 m + n/2) / n) for m >= 0
          while (-4 * m - k * n > n / 2) ++k;
          while (-4 * m - k * n < -(n / 2)) --k;
          const long long e = -4 * m - k * n;             // reduced angle 2 pi e / (4 n)
          double cc, ss;
          cis(e, 4LL * n, &cc, &ss);
          c[r] = cc;
          t[r] = ss / cc;
          kp |= (int)(((k % 4) + 4) % 4) << (2 * (r - 1));
        }
        double* rec = &tt[(size_t)tto[st] + (size_t)RS * jm];
        if (R == 5) {
          rec[0] = t[1]; rec[1] = t[2]; rec[2] = t[3]; rec[3] = t[4];
          rec[4] = c[4] / c[1]; rec[5] = c[3] / c[2];
          rec[6] = c[1]; rec[7] = c[2];
          rec[8] = C1 * c[1]; rec[9] = C2 * c[2]; rec[10] = C2 * c[1]; rec[11] = C1 * c[2];
          rec[12] = S1 * c[1]; rec[13] = S2 * c[2]; rec[14] = S2 * c[1]; rec[15] = S1 * c[2];
        } else if (R == 4) {
          rec[0] = t[1]; rec[1] = t[2]; rec[2] = t[3]; rec[3] = c[1]; rec[4] = c[2]; rec[5] = c[3] / c[1];
        } else if (R == 3) {
          rec[0] = t[1]; rec[1] = t[2]; rec[2] = c[1]; rec[3] = c[2] / c[1]; rec[4] = 0.5 * c[1];
          rec[5] = 0.86602540378443864676 * c[1];
        } else if (R == 2) {
          rec[0] = t[1]; rec[1] = c[1];
        }
        tk[toff[st] + jm] = kp;
      }
    }
    Ns *= R;
  }
}

// ------------------------------------------------------------- layout
struct Carver {
  size_t off = 0;
  char* base = nullptr;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

struct Group {
  int nx, ny, nz;
  std::vector<int> members;  // global member ids
  GroupDev d{};
  HostPlan hp[7];            // M, Mx, nx, Pu, Me, Mz, nz
  HostPlan hpn;              // M with radices up to 5 (mixed groups: the mean column)
};

int check_params(const ptt_params& p) {
  if (p.nz != 1 && (p.nz < 4 || p.nz > 512 || (p.nz & 1) || !smooth13(p.nz))) return PTT_EINVAL;
  if (p.nz > 1 && !(p.lz > 0)) return PTT_EINVAL;
  if (p.precision != PTT_FP64 && p.precision != PTT_MIXED && p.precision != PTT_MIXED_TC &&
      p.precision != PTT_FP64_DS)
    return PTT_ENOTSUP;
  if (p.nx < 8 || p.nx > 512 || (p.nx & 1) || !smooth13(p.nx)) return PTT_EINVAL;
  if (p.ny < 9 || p.ny > 513 || !smooth13(p.ny - 1)) return PTT_EINVAL;
  if (!(p.lx > 0) || !(p.re > 0) || !(p.wi > 0) || !(p.dt > 0)) return PTT_EINVAL;
  if (!(p.beta > 0 && p.beta <= 1) || !(p.eps >= 0) || !(p.kappa >= 0)) return PTT_EINVAL;
  return PTT_OK;
}

// Sizes of one shape.  Padded y grid: M Gauss points, M even, M 5-smooth
// (one FFT of length M per column), M >= (3 ny - 2)/2 so that quadratic
// products are alias-free for the retained Chebyshev modes (T_k aliases to
// -T_{2M-k} on the Gauss points).  Diagnostic grid for the energy: Me >= 2 ny - 1
// Gauss points (Fejer's first rule is exact to degree Me - 1 >= 2 ny - 2).
void group_sizes(int nx, int ny, int nz, Group& g) {
  GroupDev& d = g.d;
  d.nx = nx;
  d.K = nx / 2;
  d.N = ny;
  d.nz = nz;
  d.KZ = d.K * nz;
  d.Mz = (nz > 1) ? next_smooth(3 * nz / 2 - 2) : 1;
  d.Mx = next_smooth(3 * nx / 2 - 2);
  d.invMx = 1.0 / d.Mx;
  d.invMxf = (float)d.invMx;
  int M = (3 * ny - 2 + 1) / 2;
  while ((M & 1) || !smooth235(M)) ++M;
  d.M = M;
  d.P = M;
  d.Pu = 2 * (ny - 1);
  int Me = 2 * ny - 1;
  while ((Me & 1) || !smooth235(Me)) ++Me;
  d.Me = Me;
  const size_t target = 96 * 1024;
  auto cols = [&](int P) {
    long long c = (long long)(target / smem_ycols(1, P, 0));
    if (c < 1) c = 1;
    if (c > 16) c = 16;
    return (int)c;
  };
  d.Ccol = cols(d.M);
  d.CcolE = cols(d.Me);
  d.CcolU = cols(d.Pu);
  d.xthreads = 512;   // launch-shape defaults (ptt_autotune may change them)
  d.zC = 8;
  g.hp[0] = make_plan(d.M);
  g.hp[1] = make_plan(d.Mx, true);
  g.hp[2] = make_plan(nx);
  g.hp[3] = make_plan(d.Pu);
  g.hp[4] = make_plan(d.Me);
  g.hp[5] = make_plan(d.Mz, true);
  g.hp[6] = make_plan(nz);
}

// The plans of an FP32 group with radix-8 passes: those of the padded
// lengths (M, Mx, Mz) and of the energy grid (Me), which only FP32 kernels
// use in such groups.  The unpadded lengths (nx, 2 (ny - 1), nz) keep radices
// up to 5 (and 7, 11, 13): the FP64 state transforms (set and get state, the
// x synthesis of Tr c) and the double-single Tr c transforms use them.
void wide_plans(Group& g) {
  const int n[7] = {g.d.M, g.d.Mx, g.d.nx, g.d.Pu, g.d.Me, g.d.Mz, g.d.nz};
  const bool three[7] = {false, true, false, false, false, true, false};
  const bool widen[7] = {true, true, false, false, true, true, false};
  for (int i = 0; i < 7; ++i)
    if (widen[i]) g.hp[i] = make_plan(n[i], three[i], true);
}

// Carve (or, with base == nullptr, size) all device arrays.
void carve(std::vector<Group>& groups, Carver& cv) {
  for (Group& g : groups) {
    GroupDev& d = g.d;
    const int nb = (int)g.members.size();
    d.nb = nb;
    // columns per block: fit the shared-memory target, but leave at least
    // about two blocks per SM (152 SMs) for the column counts of each pass
    auto cap = [&](int c, int nfields) {
      const int want = (int)((long long)d.KZ * nfields * nb / 304);
      return std::max(1, std::min(c, want));
    };
    d.Ccol = cap(d.Ccol, 9);
    d.CcolE = cap(d.CcolE, 2);
    d.CcolU = cap(d.CcolU, 1);
    const bool d3 = d.nz > 1;
    const size_t nf = d3 ? 9 : 5, ne = d3 ? 8 : 4;   // state fields, evolved quantities
    const size_t NK = (size_t)d.N * d.KZ, rows = (size_t)d.M, Je = (size_t)d.Me;
    const size_t KZ = d.KZ, K = d.K, nzz = d.nz;
    d.prm = cv.take<MemberPrm>(nb);
    d.status = cv.take<int>(nb);
    d.count = cv.take<long long>(nb);
    d.X = cv.take<double2>((size_t)nb * nf * NK);
    d.Eh = cv.take<double2>((size_t)4 * nb * ne * NK);
    d.Nh = cv.take<double2>((size_t)4 * nb * ne * NK);
    d.Yp = d.Zp = nullptr;
    d.Ypf = d.Zpf = nullptr;
    d.Y3 = d.Z3 = d.W3 = d.V3 = nullptr;
    d.Y3f = d.Z3f = d.W3f = d.V3f = nullptr;
    if (!d3) {
      if (d.f32) {
        d.Ypf = cv.take<float2>((size_t)nb * 9 * rows * K);
        d.Zpf = cv.take<float2>((size_t)nb * 5 * rows * K);
      } else {
        d.Yp = cv.take<double2>((size_t)nb * 9 * rows * K);
        d.Zp = cv.take<double2>((size_t)nb * 5 * rows * K);
      }
    } else {
      const size_t yp = rows * KZ, zp = rows * d.Mz * K;
      if (d.f32) {
        d.Y3f = cv.take<float2>((size_t)nb * 17 * yp);
        d.Z3f = cv.take<float2>((size_t)nb * 26 * zp);
        d.W3f = cv.take<float2>((size_t)nb * 9 * zp);
        d.V3f = cv.take<float2>((size_t)nb * 9 * yp);
      } else {
        d.Y3 = cv.take<double2>((size_t)nb * 17 * yp);
        d.Z3 = cv.take<double2>((size_t)nb * 26 * zp);
        d.W3 = cv.take<double2>((size_t)nb * 9 * zp);
        d.V3 = cv.take<double2>((size_t)nb * 9 * yp);
      }
    }
    d.Ym = d.f32 ? cv.take<double2>((size_t)nb * (d3 ? 17 : 9) * rows) : nullptr;
    d.Zm = d.f32 ? cv.take<double2>((size_t)nb * nf * rows) : nullptr;
    d.NR = cv.take<double2>((size_t)nb * nf * NK);
    d.Rb = cv.take<double2>((size_t)nb * 4 * NK);
    d.SS = d3 ? cv.take<double2>((size_t)nb * spec3_scratch_columns() * NK) : nullptr;
    d.qt = cv.take<double>((size_t)nb * 4 * 3 * 3 * NK);
    d.qtG = cv.take<double>((size_t)nb * 4 * 3 * 2 * KZ);
    d.vh = cv.take<double>((size_t)nb * 4 * NK);
    d.vhS = cv.take<double>((size_t)nb * 4 * 2 * KZ);
    d.wrow = cv.take<double>((size_t)3 * d.N);
    d.ccw = cv.take<double>(Je);
    d.DY = cv.take<double2>((size_t)nb * (d3 ? 3 : 2) * Je * KZ);
    d.DT = cv.take<double2>((size_t)nb * NK);
    d.DV = cv.take<double>((size_t)nb * d.N * nzz * d.nx);
    d.ntile = diag_tiles(d.N, d.nx, d.nz);
    d.part = cv.take<double>((size_t)nb * d.ntile * kPart);
    d.DM = cv.take<double2>((size_t)nb * (d3 ? 8 : 4) * KZ);
    d.DZ = d3 ? cv.take<double2>(std::max((size_t)nb, (size_t)9) * d.N * nzz * K) : nullptr;
    d.DMZ = d3 ? cv.take<double2>((size_t)nb * 8 * nzz * K) : nullptr;
    d.MV = d3 ? cv.take<double>((size_t)nb * 8 * nzz * d.nx) : nullptr;
    d.ring = cv.take<ptt_diag>((size_t)nb * kRing);
    d.hist = cv.take<unsigned long long>((size_t)nb * 8 * (PTT_HIST_BINS + 2));
    d.hrange = cv.take<double>((size_t)nb * 16);
    d.macc = cv.take<double>((size_t)nb * kMacc);
    d.statout = cv.take<double>((size_t)kMacc);
    // mixed groups: pre-split tables of the tensor-core Chebyshev passes
    const bool mma = d.f32 && d.ymma && cheb_mma_supported(d.M, d.N);
    d.Wyi = mma ? cv.take<uint16_t>(cheb_mma_table_bytes(d.M, d.N, 1) / 2) : nullptr;
    d.Wyf = mma ? cv.take<uint16_t>(cheb_mma_table_bytes(d.M, d.N, 0) / 2) : nullptr;
    d.mma_err = cv.take<int>(1);
    d.ymma = mma ? 1 : 0;
    d.stage = cv.take<double>((size_t)nf * d.N * nzz * d.nx);
    d.stageS = cv.take<double2>((size_t)nf * NK);
    FftPlan* pls[7] = {&d.plP, &d.plMx, &d.plNx, &d.plPu, &d.plPe, &d.plMz, &d.plNz};
    for (int i = 0; i < 7; ++i) {
      pls[i]->n = g.hp[i].n;
      pls[i]->nst = (int)g.hp[i].radix.size();
      for (int s = 0; s < pls[i]->nst; ++s) pls[i]->radix[s] = g.hp[i].radix[s];
      plan_pass_consts(*pls[i]);
      pls[i]->tw = cv.take<double2>((size_t)g.hp[i].n);
      // single-precision tables: the step's padded lengths and the energy grid
      pls[i]->twf = (d.f32 && (i < 2 || i == 4 || i == 5)) ? cv.take<float2>((size_t)g.hp[i].n) : nullptr;
      // double-single tables: every length of a double-single group; the
      // unpadded y and z lengths of a mixed group (its Tr c transforms)
      pls[i]->twd = (d.ds || (d.f32 && (i == 0 || i == 3 || i == 6))) ? cv.take<float4>((size_t)g.hp[i].n)
                                                                   : nullptr;
      int nrec = 0, ndbl = 0;
      tangent_offsets(g.hp[i], pls[i]->toff, pls[i]->tto, &nrec, &ndbl);
      pls[i]->tt = cv.take<double>((size_t)ndbl);
      pls[i]->tk = cv.take<int>((size_t)nrec);
    }
    d.tw4P = cv.take<double2>((size_t)d.M);
    d.tw4Pf = d.f32 ? cv.take<float2>((size_t)d.M) : nullptr;
    d.tw4Pi = cv.take<double2>((size_t)d.M);
    d.tw4Pif = d.f32 ? cv.take<float2>((size_t)d.M) : nullptr;
    d.tw4E = cv.take<double2>((size_t)d.Me);
    d.tw4Ef = d.f32 ? cv.take<float2>((size_t)d.Me) : nullptr;
    d.tw4Pd = (d.ds || d.f32) ? cv.take<float4>((size_t)d.M) : nullptr;
    d.tw4Pid = (d.ds || d.f32) ? cv.take<float4>((size_t)d.M) : nullptr;
    // mixed groups: the narrow plan of M shares plP's tables
    d.plPn = d.plP;
    if (d.f32) {
      d.plPn.nst = (int)g.hpn.radix.size();
      for (int s = 0; s < d.plPn.nst; ++s) d.plPn.radix[s] = g.hpn.radix[s];
      plan_pass_consts(d.plPn);
    }
    d.tw4Ed = d.ds ? cv.take<float4>((size_t)d.Me) : nullptr;
  }
}

std::vector<Group> make_groups(const ptt_params* pm, int nmem) {
  std::map<std::tuple<int, int, int, int>, int> idx;
  std::vector<Group> groups;
  for (int i = 0; i < nmem; ++i) {
    auto key = std::make_tuple(pm[i].nx, pm[i].ny, pm[i].nz, pm[i].precision);
    auto it = idx.find(key);
    if (it == idx.end()) {
      idx[key] = (int)groups.size();
      Group g;
      g.nx = pm[i].nx;
      g.ny = pm[i].ny;
      g.nz = pm[i].nz;
      group_sizes(g.nx, g.ny, g.nz, g);
      g.d.f32 = (pm[i].precision == PTT_MIXED || pm[i].precision == PTT_MIXED_TC) ? 1 : 0;
      g.d.ds = (pm[i].precision == PTT_FP64_DS) ? 1 : 0;
      if (g.d.f32) { g.hpn = g.hp[0]; wide_plans(g); }
      g.d.ymma = (pm[i].precision == PTT_MIXED_TC) ? 1 : 0;   // requested; carve() checks the shape
      groups.push_back(std::move(g));
      it = idx.find(key);
    }
    groups[it->second].members.push_back(i);
  }
  return groups;
}

// A context can take one launch per stage over all its groups when they
// are all 2D, of one precision, without tensor-core passes, 2 to
// multi2d_max_groups() of them.
bool multi_eligible(const std::vector<Group>& groups) {
  if (groups.size() < 2 || (int)groups.size() > multi2d_max_groups()) return false;
  for (const Group& g : groups)
    if (g.d.nz != 1 || g.d.ymma || g.d.f32 != groups[0].d.f32 || g.d.ds != groups[0].d.ds) return false;
  return true;
}

}  // namespace

struct ptt_ctx {
  std::vector<ptt_params> prm;
  std::vector<Group> groups;
  std::vector<std::pair<int, int>> where;  // member -> (group, index in group)
  std::vector<long long> last_read;        // last diagnostics step returned
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  // step graphs (see capture_step_graph): 0 first step of a ptt_step call,
  // 1 later steps, 2 diagnostics of the last step
  cudaGraph_t graph[3] = {nullptr, nullptr, nullptr};
  cudaGraphExec_t exec[3] = {nullptr, nullptr, nullptr};
  std::vector<cudaStream_t> gstreams;  // one capture branch per group
  std::vector<cudaStream_t> dstreams;  // the group's diagnostics branch
  std::vector<cudaStream_t> pstreams;  // [2 per group] its energy and mid-plane parts
  std::vector<cudaEvent_t> gevents;
  std::vector<cudaEvent_t> devents;
  std::vector<cudaEvent_t> pevents;    // [3 per group] fork / join of those parts
  int launches = 0;
  int device = 0;
  double timeout_s = 3600.0;           // wall-clock limit of ptt_synchronize (<= 0: none)
  // launch mode of the step graphs: 0 one branch per shape group, 1 one
  // launch per kernel of each stage over all groups (2D contexts)
  int launch_mode = 0;
  void* multi_dev = nullptr;           // workspace region of the plan (null: not eligible)
  Multi2DPlan* multi = nullptr;
};

thread_local char g_last_error[512] = "";

int fail_cuda(cudaError_t e, const char* what, int line) {
  std::snprintf(g_last_error, sizeof(g_last_error), "%s (line %d): %s", what, line,
                cudaGetErrorString(e));
  return PTT_ECUDA;
}

#define CK(x)                                             \
  do {                                                    \
    cudaError_t e_ = (x);                                 \
    if (e_ != cudaSuccess) return fail_cuda(e_, #x, __LINE__); \
  } while (0)

// ---------------------------------------------------------------------------
// Host helpers shared with the workspace-free entry point (ptt_noalloc.cu).
namespace ptt {

void set_last_error(const char* msg) {
  std::snprintf(g_last_error, sizeof(g_last_error), "%s", msg);
}

int shape_plan(const ptt_params& p, GroupDev& d, std::vector<double2>& twP,
               std::vector<double2>& twMx, std::vector<double2>& tw4, MemberPrm& prm,
               std::vector<double>* tt, std::vector<int>* tk) {
  const int s = check_params(p);
  if (s) return s;
  if (p.precision != PTT_FP64) return PTT_ENOTSUP;
  if (p.nz != 1) return PTT_ENOTSUP;
  Group g;
  g.nx = p.nx;
  g.ny = p.ny;
  g.nz = 1;
  group_sizes(p.nx, p.ny, 1, g);
  d = g.d;
  d.nb = 1;
  // columns per block as carve() caps them for one member
  d.Ccol = std::max(1, std::min(d.Ccol, (int)((long long)d.KZ * 9 / 304)));
  FftPlan* pls[2] = {&d.plP, &d.plMx};
  std::vector<double2>* tws[2] = {&twP, &twMx};
  for (int i = 0; i < 2; ++i) {
    const HostPlan& hp = g.hp[i];
    pls[i]->n = hp.n;
    pls[i]->nst = (int)hp.radix.size();
    for (int k = 0; k < pls[i]->nst; ++k) pls[i]->radix[k] = hp.radix[k];
    plan_pass_consts(*pls[i]);
    // tangent-form twiddle records of the FP64 passes (device pointers are
    // set by the caller once the tables have a home)
    int nrec = 0, ndbl = 0;
    tangent_offsets(hp, pls[i]->toff, pls[i]->tto, &nrec, &ndbl);
    tangent_tables(hp, tt[i], tk[i]);
    tws[i]->resize(hp.n);
    for (int k = 0; k < hp.n; ++k) {
      double cc, ss;
      cis(k, hp.n, &cc, &ss);
      (*tws[i])[k] = make_double2(cc, -ss);
    }
  }
  // tw4: the forward table of the Gauss-grid transforms, then the inverse one
  std::vector<double2> inv;
  quarter_tables(d.M, tw4, inv);
  tw4.insert(tw4.end(), inv.begin(), inv.end());
  member_prm(p, prm);
  return PTT_OK;
}

void plan_pass_consts(FftPlan& pl) {
  // the same multiply-high reciprocal as the device's fast_div
  auto magic = [](unsigned d) { return d == 1u ? 0u : 0xFFFFFFFFu / d + 1u; };
  int Ns = 1;
  for (int s = 0; s < pl.nst; ++s) {
    const int R = pl.radix[s];
    pl.pnb[s] = pl.n / R;
    pl.pst[s] = pl.n / (Ns * R);
    pl.pns[s] = Ns;
    pl.pmb[s] = magic((unsigned)pl.pnb[s]);
    pl.pms[s] = magic((unsigned)Ns);
    Ns *= R;
  }
}

void member_prm(const ptt_params& p, MemberPrm& q) {
  q.lx = p.lx; q.lz = (p.nz > 1) ? p.lz : 1.0;
  q.re = p.re; q.wi = p.wi; q.beta = p.beta; q.eps = p.eps;
  q.kappa = p.kappa; q.dt = p.dt;
  q.inv_wi = 1.0 / p.wi;
  q.gam = (1.0 - p.beta) / (p.re * p.wi);
  q.nu = p.beta / p.re;
  q.forcing = 2.0 / p.re;
  q.trc_max = p.blowup_trc_max > 0 ? p.blowup_trc_max : 1e300;
  q.u_max = p.blowup_u_max > 0 ? p.blowup_u_max : 1e300;
  q.kx1 = 2.0 * kPi / q.lx;
  q.kz1 = 2.0 * kPi / q.lz;
  q.kx1f = (float)q.kx1;
  q.kz1f = (float)q.kz1;
  q.epsf = (float)q.eps;
  q.inv_wif = (float)q.inv_wi;
}

}  // namespace ptt

extern "C" {

int ptt_workspace_size(const ptt_params* pm, int32_t nmem, size_t* bytes) {
  if (!pm || nmem <= 0 || !bytes) return PTT_EINVAL;
  for (int i = 0; i < nmem; ++i) {
    int s = check_params(pm[i]);
    if (s) return s;
  }
  std::vector<Group> groups = make_groups(pm, nmem);
  for (Group& g : groups) {
    if (g.d.nz == 1 && (smem_xfused(g.d.Mx, g.d.f32) > 227 * 1024 || smem_spec(g.d.N) > 227 * 1024))
      return PTT_EINVAL;
    if (g.d.nz > 1 && smem_xfused3(g.d.Mx, g.d.f32) == 0)
      return PTT_EINVAL;
  }
  Carver cv;
  carve(groups, cv);
  if (multi_eligible(groups)) cv.take<char>(multi2d_bytes((int)groups.size()));
  *bytes = cv.off + 256;
  return PTT_OK;
}

// The step as CUDA graphs, one branch per shape group (a fork per group from
// the capture stream, a join back; re-capturing replaces existing graphs).  The diagnostics of a
// state only read it (and write their own buffers), and only the spectral
// stage of the next step overwrites it, so they run beside the next step's
// transforms (stages 0-2) on a second branch per group that the spectral
// stage waits for.  Graph 0 is the first step of a ptt_step call (stages 0-3;
// the state it starts from was diagnosed when it was made), graph 1 a later
// step (the previous step's diagnostics beside stages 0-2, then stage 3), and
// graph 2 the diagnostics of the last step's result (stage 4).  Within the
// diagnostics, the energy transform and the mid-plane sums run on branches of
// their own beside the Tr c chain (launch_diag_split).
// The same with one launch per kernel and stage over all groups (launch
// mode 1): the diagnostics of the previous step on one branch beside the
// next step's transforms.
static cudaError_t capture_kind_multi(ptt_ctx* c, int kind, int* nl) {
  const Multi2DPlan* p = c->multi;
  auto diag = [&](cudaStream_t s0) {
    const DiagStreams d{{s0, c->pstreams[0], c->pstreams[1]}, {c->pevents[0], c->pevents[1], c->pevents[2]}};
    return launch_diag_multi(p, d, nl);
  };
  if (kind == 2) return diag(c->cap);
  cudaError_t le = cudaSuccess;
  cudaStream_t ds = c->dstreams[0];
  if (kind == 1) {
    le = cudaEventRecord(c->gevents.back(), c->cap);
    if (!le) le = cudaStreamWaitEvent(ds, c->gevents.back(), 0);
    if (!le) le = diag(ds);
    if (!le) le = cudaEventRecord(c->devents[0], ds);
  }
  for (int s = 0; s < 3 && !le; ++s) le = launch_stage_multi(p, s, c->cap, nl);
  if (!le && kind == 1) le = cudaStreamWaitEvent(c->cap, c->devents[0], 0);
  if (!le) le = launch_stage_multi(p, 3, c->cap, nl);
  return le;
}

static cudaError_t capture_kind(ptt_ctx* c, int kind, int* nl) {
  if (c->launch_mode == 1) return capture_kind_multi(c, kind, nl);
  cudaError_t le = cudaEventRecord(c->gevents.back(), c->cap);
  for (size_t gi = 0; gi < c->groups.size() && !le; ++gi) {
    cudaStream_t gs = c->gstreams[gi], ds = c->dstreams[gi];
    const GroupDev& gd = c->groups[gi].d;
    const bool d3 = gd.nz > 1;
    le = cudaStreamWaitEvent(gs, c->gevents.back(), 0);
    auto diag = [&](cudaStream_t s0) {
      const DiagStreams d{{s0, c->pstreams[2 * gi], c->pstreams[2 * gi + 1]},
                          {c->pevents[3 * gi], c->pevents[3 * gi + 1], c->pevents[3 * gi + 2]}};
      return d3 ? launch_diag_split3(gd, d, nl) : launch_diag_split(gd, d, nl);
    };
    if (!le && kind == 1) {
      le = cudaStreamWaitEvent(ds, c->gevents.back(), 0);
      if (!le) le = diag(ds);
      if (!le) le = cudaEventRecord(c->devents[gi], ds);
    }
    if (kind == 2) {
      if (!le) le = diag(gs);
    } else {
      for (int s = 0; s < 3 && !le; ++s) le = d3 ? launch_stage3(gd, s, gs, nl) : launch_stage(gd, s, gs, nl);
      if (!le && kind == 1) le = cudaStreamWaitEvent(gs, c->devents[gi], 0);
      if (!le) le = d3 ? launch_stage3(gd, 3, gs, nl) : launch_stage(gd, 3, gs, nl);
    }
    if (!le) le = cudaEventRecord(c->gevents[gi], gs);
    if (!le) le = cudaStreamWaitEvent(c->cap, c->gevents[gi], 0);
  }
  return le;
}

static int capture_step_graph(ptt_ctx* c) {
  for (int k = 0; k < 3; ++k) {
    if (c->exec[k]) { cudaGraphExecDestroy(c->exec[k]); c->exec[k] = nullptr; }
    if (c->graph[k]) { cudaGraphDestroy(c->graph[k]); c->graph[k] = nullptr; }
  }
  if (c->multi) { multi2d_destroy(c->multi); c->multi = nullptr; }
  if (c->launch_mode == 1) {
    // the plan copies the groups as they are now (launch shapes included)
    std::vector<const GroupDev*> gs;
    for (const Group& g : c->groups) gs.push_back(&g.d);
    cudaError_t e = cudaSuccess;
    c->multi = multi2d_create(gs, c->multi_dev, c->stream, &e);
    if (!c->multi) return fail_cuda(e ? e : cudaErrorInvalidValue, "multi2d_create", __LINE__);
  }
  for (int k = 0; k < 3; ++k) {
    CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
    int nl = 0;
    const cudaError_t le = capture_kind(c, k, &nl);
    const cudaError_t ee = cudaStreamEndCapture(c->cap, &c->graph[k]);
    if (le) return fail_cuda(le, "launch during graph capture", __LINE__);
    if (ee) return fail_cuda(ee, "cudaStreamEndCapture", __LINE__);
    CK(cudaGraphInstantiate(&c->exec[k], c->graph[k], 0));
    if (k == 1) c->launches = nl;   // every kernel of one step, diagnostics included
  }
  return PTT_OK;
}

int ptt_create(const ptt_params* pm, int32_t nmem, void* d_ws, size_t bytes, void* stream,
               ptt_ctx** out) {
  if (!out) return PTT_EINVAL;
  *out = nullptr;
  size_t need = 0;
  int s = ptt_workspace_size(pm, nmem, &need);
  if (s) return s;
  if (!d_ws || ((uintptr_t)d_ws & 255)) return PTT_EINVAL;
  if (bytes < need) return PTT_ENOMEM;
  std::unique_ptr<ptt_ctx> c(new (std::nothrow) ptt_ctx());
  if (!c) return PTT_ENOMEM;
  c->prm.assign(pm, pm + nmem);
  c->groups = make_groups(pm, nmem);
  c->stream = (cudaStream_t)stream;
  CK(cudaGetDevice(&c->device));
  Carver cv;
  cv.base = (char*)d_ws;
  carve(c->groups, cv);
  if (multi_eligible(c->groups)) c->multi_dev = cv.take<char>(multi2d_bytes((int)c->groups.size()));
  c->where.assign(nmem, {0, 0});
  c->last_read.assign(nmem, -1);
  int optin = 0;
  CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
  for (Group& g : c->groups) {
    if (g.d.nz == 1 && (smem_xfused(g.d.Mx, g.d.f32) > (size_t)optin || smem_spec(g.d.N) > (size_t)optin))
      return PTT_EINVAL;
    if (g.d.nz > 1 && (smem_xfused3(g.d.Mx, g.d.f32) == 0 || smem_xfused3(g.d.Mx, g.d.f32) > (size_t)optin))
      return PTT_EINVAL;
  }
  CK(set_kernel_attributes(optin));
  CK(set_kernel_attributes3(optin));
  CK(set_cheb_mma_attributes(optin));
  int nsm = 0;
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
  CK(cudaMemsetAsync(d_ws, 0, need - 256, c->stream));
  for (size_t gi = 0; gi < c->groups.size(); ++gi) {
    Group& g = c->groups[gi];
    GroupDev& d = g.d;
    const int nb = d.nb, N = d.N, K = d.KZ, nzz = d.nz;   // K: modes per Chebyshev index
    const size_t NK = (size_t)N * K;
    for (int i = 0; i < nb; ++i) c->where[g.members[i]] = {(int)gi, i};
    d.nsm = nsm;
    if (d.Wyi) {
      for (int inv = 0; inv < 2; ++inv) {
        std::vector<uint16_t> tab;
        cheb_mma_tables(d.M, d.N, 1 - inv, tab);
        CK(cudaMemcpyAsync((void*)(inv ? d.Wyf : d.Wyi), tab.data(), tab.size() * sizeof(uint16_t),
                           cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
      }
    }
    // member parameters
    std::vector<MemberPrm> mp(nb);
    for (int i = 0; i < nb; ++i) {
      member_prm(pm[g.members[i]], mp[i]);
    }
    CK(cudaMemcpyAsync(d.prm, mp.data(), nb * sizeof(MemberPrm), cudaMemcpyHostToDevice, c->stream));
    // row weights of the quasi-tridiagonal form
    std::vector<double> w(3 * (size_t)N, 0.0);
    for (int n = 2; n < N; ++n) {
      w[n] = 1.0 / (4.0 * n * (n - 1));
      w[N + n] = 1.0 / (2.0 * ((double)n * n - 1.0));
      w[2 * N + n] = 1.0 / (4.0 * n * (n + 1));
    }
    // operator tables per member, SBDF order, system, mode, parity
    std::vector<double> qt((size_t)nb * 4 * 3 * 3 * NK, 0.0), qtG((size_t)nb * 4 * 3 * 2 * K, 0.0);
    std::vector<double> vh((size_t)nb * 4 * NK, 0.0), vhS((size_t)nb * 4 * 2 * K, 0.0);
    std::vector<double> phi(N), rz(N, 0.0);
    for (int i = 0; i < nb; ++i) {
      const ptt_params& p = pm[g.members[i]];
      const double nu = p.beta / p.re;
      for (int o = 0; o < 4; ++o) {
        const double a0dt = kSA0[o] / p.dt;
        for (int m = 0; m < K; ++m) {
          // mode m = mx * nz + mz, mz in FFT order (signed wavenumber)
          const int mx = m / nzz, mzi = m - mx * nzz;
          const int sz = (mzi < nzz / 2) ? mzi : mzi - nzz;
          const double kxm = 2.0 * kPi * mx / p.lx;
          const double kzm = (nzz > 1) ? 2.0 * kPi * sz / p.lz : 0.0;
          const double k2 = kxm * kxm + kzm * kzm;
          const double al[3] = {a0dt + p.kappa * k2, a0dt + nu * k2, k2};
          const double be[3] = {p.kappa, nu, 1.0};
          for (int ts = 0; ts < 3; ++ts) {
            if (ts == 0 && p.kappa == 0.0) continue;
            if (ts == 2 && m == 0) continue;
            double* base = &qt[((((size_t)i * 4 + o) * 3 + ts) * 3) * NK + (size_t)m * N];
            for (int par = 0; par < 2; ++par) {
              qt_tables(N, al[ts], be[ts], w.data(), w.data() + N, w.data() + 2 * N, par, base,
                        base + NK, base + 2 * NK,
                        &qtG[((((size_t)i * 4 + o) * 3 + ts) * 2 + par) * K + m], 1);
            }
          }
          if (m == 0) continue;
          // homogeneous solutions of the influence-matrix step:
          // phi_h: rows of (alpha - nu D^2) phi = 0 with the parity sum = 1,
          // v_h: rows of (k^2 - D^2) v = -phi_h with the parity sum = 0.
          const double* T1 = &qt[((((size_t)i * 4 + o) * 3 + 1) * 3) * NK + (size_t)m * N];
          const double* T2 = &qt[((((size_t)i * 4 + o) * 3 + 2) * 3) * NK + (size_t)m * N];
          double* vo = &vh[((size_t)i * 4 + o) * NK + (size_t)m * N];
          for (int par = 0; par < 2; ++par) {
            const double G1 = qtG[((((size_t)i * 4 + o) * 3 + 1) * 2 + par) * K + m];
            const double G2 = qtG[((((size_t)i * 4 + o) * 3 + 2) * 2 + par) * K + m];
            std::vector<double> vv(N, 0.0);
            std::fill(phi.begin(), phi.end(), 0.0);
            qt_solve_host(N, par, al[1], rz.data(), phi.data(), T1, T1 + NK, T1 + 2 * NK, G1,
                          w.data(), w.data() + N, w.data() + 2 * N, 1.0, 1.0, 1);
            qt_solve_host(N, par, al[2], phi.data(), vv.data(), T2, T2 + NK, T2 + 2 * NK, G2,
                          w.data(), w.data() + N, w.data() + 2 * N, 0.0, -1.0, 1);
            double S = 0.0;
            for (int n = par; n < N; n += 2) {
              vo[n] = vv[n];
              S += (double)n * n * vv[n];
            }
            vhS[(((size_t)i * 4 + o) * 2 + par) * K + m] = 1.0 / S;
          }
        }
      }
    }
    CK(cudaMemcpyAsync((void*)d.qt, qt.data(), qt.size() * 8, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync((void*)d.qtG, qtG.data(), qtG.size() * 8, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync((void*)d.vh, vh.data(), vh.size() * 8, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync((void*)d.vhS, vhS.data(), vhS.size() * 8, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync((void*)d.wrow, w.data(), w.size() * 8, cudaMemcpyHostToDevice, c->stream));
    // Fejer's first rule on the Me Gauss points y_j = cos(theta_j),
    // theta_j = pi (2j+1)/(2 Me): w_j = int of the interpolant's basis,
    // w_j = (2/Me) [1 + sum_{n even, 2 <= n < Me} cos(n theta_j) * 2/(1 - n^2)]
    {
      const int Me = d.Me;
      std::vector<double> cw(Me, 0.0);
      for (int j = 0; j < Me; ++j) {
        double acc = 1.0;
        for (int n = 2; n < Me; n += 2) {
          double cc, ss;
          cis((long long)n * (2 * j + 1), 4LL * Me, &cc, &ss);
          acc += cc * 2.0 / (1.0 - (double)n * n);
        }
        cw[j] = 2.0 / Me * acc;
      }
      CK(cudaMemcpyAsync((void*)d.ccw, cw.data(), cw.size() * 8, cudaMemcpyHostToDevice, c->stream));
    }
    // quarter-period twiddles of the Gauss-grid transforms (forward and
    // inverse on the padded grid, inverse on the diagnostic grid)
    {
      std::vector<double2> fwd, inv, fwdE, invE;
      quarter_tables(d.M, fwd, inv);
      quarter_tables(d.Me, fwdE, invE);
      const std::vector<double2>* src[3] = {&fwd, &inv, &invE};
      const double2* dst[3] = {d.tw4P, d.tw4Pi, d.tw4E};
      const float2* dstf[3] = {d.tw4Pf, d.tw4Pif, d.tw4Ef};
      const float4* dstd[3] = {d.tw4Pd, d.tw4Pid, d.tw4Ed};
      std::vector<float2> twf[3];
      std::vector<float4> twd[3];
      for (int t = 0; t < 3; ++t) {
        const std::vector<double2>& tw = *src[t];
        CK(cudaMemcpyAsync((void*)dst[t], tw.data(), tw.size() * sizeof(double2), cudaMemcpyHostToDevice,
                           c->stream));
        if (dstf[t]) {
          twf[t].resize(tw.size());
          for (size_t k = 0; k < tw.size(); ++k) twf[t][k] = make_float2((float)tw[k].x, (float)tw[k].y);
          CK(cudaMemcpyAsync((void*)dstf[t], twf[t].data(), twf[t].size() * sizeof(float2),
                             cudaMemcpyHostToDevice, c->stream));
        }
        if (dstd[t]) {
          twd[t].resize(tw.size());
          for (size_t k = 0; k < tw.size(); ++k) twd[t][k] = ds_split(tw[k]);
          CK(cudaMemcpyAsync((void*)dstd[t], twd[t].data(), twd[t].size() * sizeof(float4),
                             cudaMemcpyHostToDevice, c->stream));
        }
      }
      CK(cudaStreamSynchronize(c->stream));
    }
    // twiddle tables
    FftPlan* pls[7] = {&d.plP, &d.plMx, &d.plNx, &d.plPu, &d.plPe, &d.plMz, &d.plNz};
    for (int t = 0; t < 7; ++t) {
      const int n = pls[t]->n;
      std::vector<double2> tw(n);
      for (int k = 0; k < n; ++k) {
        double cc, ss;
        cis(k, n, &cc, &ss);
        tw[k] = make_double2(cc, -ss);
      }
      CK(cudaMemcpyAsync((void*)pls[t]->tw, tw.data(), n * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
      {
        std::vector<double> tt;
        std::vector<int> tk;
        tangent_tables(g.hp[t], tt, tk);
        CK(cudaMemcpyAsync((void*)pls[t]->tt, tt.data(), tt.size() * sizeof(double),
                           cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync((void*)pls[t]->tk, tk.data(), tk.size() * sizeof(int),
                           cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
      }
      if (pls[t]->twf) {
        std::vector<float2> twf(n);
        for (int k = 0; k < n; ++k) twf[k] = make_float2((float)tw[k].x, (float)tw[k].y);
        CK(cudaMemcpyAsync((void*)pls[t]->twf, twf.data(), n * sizeof(float2), cudaMemcpyHostToDevice,
                           c->stream));
      }
      std::vector<float4> twd;
      if (pls[t]->twd) {
        twd.resize(n);
        for (int k = 0; k < n; ++k) twd[k] = ds_split(tw[k]);
        CK(cudaMemcpyAsync((void*)pls[t]->twd, twd.data(), n * sizeof(float4), cudaMemcpyHostToDevice,
                           c->stream));
      }
      CK(cudaStreamSynchronize(c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
  }
  // capture one step of every group into a graph: the groups are
  // independent, so each gets its own branch (fork/join through events)
  CK(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
  c->gstreams.assign(c->groups.size(), nullptr);
  c->dstreams.assign(c->groups.size(), nullptr);
  c->pstreams.assign(2 * c->groups.size(), nullptr);
  c->gevents.assign(c->groups.size() + 1, nullptr);
  c->devents.assign(c->groups.size(), nullptr);
  c->pevents.assign(3 * c->groups.size(), nullptr);
  for (auto& s2 : c->gstreams) CK(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
  for (auto& s2 : c->dstreams) CK(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
  for (auto& s2 : c->pstreams) CK(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
  for (auto& e2 : c->gevents) CK(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming));
  for (auto& e2 : c->devents) CK(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming));
  for (auto& e2 : c->pevents) CK(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming));
  {
    const int s3 = capture_step_graph(c.get());
    if (s3) return s3;
  }
  *out = c.release();
  return PTT_OK;
}

int ptt_create_ensemble(const ptt_params* per_member, int32_t nmembers, void* d_workspace,
                        size_t bytes, void* cuda_stream, ptt_ctx** out) {
  return ptt_create(per_member, nmembers, d_workspace, bytes, cuda_stream, out);
}

static int member_ok(ptt_ctx* c, int member) {
  return c && member >= 0 && member < (int)c->prm.size();
}

// laminar_c: the c fields of h are the laminar state, a function of y alone;
// their coefficients at kx, kz != 0 are then set to exactly zero instead of
// the rounding residue of the x / z analysis of constant rows.
static int upload_phys(ptt_ctx* c, int member, const double* h, bool laminar_c = false) {
  auto [gi, b] = c->where[member];
  Group& g = c->groups[gi];
  const bool d3 = g.d.nz > 1;
  const int nf = d3 ? 9 : 5;
  const size_t n = (size_t)nf * g.d.N * g.d.nz * g.d.nx;
  CK(cudaMemcpyAsync(g.d.stage, h, n * 8, cudaMemcpyHostToDevice, c->stream));
  CK(d3 ? launch_phys_to_state3(g.d, b, c->stream) : launch_phys_to_state(g.d, b, c->stream));
  if (laminar_c) {
    // state [member][field][mode][n]: the non-mean modes of a field are the
    // contiguous range after mode 0
    const size_t NK = (size_t)g.d.N * g.d.KZ;
    for (int f = d3 ? 3 : 2; f < nf; ++f)
      CK(cudaMemsetAsync(g.d.X + ((size_t)b * nf + f) * NK + g.d.N, 0,
                         (NK - g.d.N) * sizeof(double2), c->stream));
  }
  CK(d3 ? launch_diag3(g.d, c->stream, nullptr) : launch_diag(g.d, c->stream, nullptr));
  CK(cudaStreamSynchronize(c->stream));
  c->last_read[member] = -1;
  return PTT_OK;
}

int ptt_init_state(ptt_ctx* c, int32_t member, uint64_t seed, double amplitude) {
  if (!member_ok(c, member) || !(amplitude >= 0)) return PTT_EINVAL;
  std::vector<double> f;
  if (c->prm[member].nz > 1) initial_fields3(c->prm[member], seed, amplitude, f);
  else initial_fields(c->prm[member], seed, amplitude, f);
  return upload_phys(c, member, f.data(), true);
}

// 3D physical values: the ABI orders them [field][z][y][x], the staging
// buffer of the transforms [field][y][z][x]; the host reorders at the
// boundary (to_staging: ABI -> staging).
static void reorder_zy(const double* src, double* dst, int nf, int ny, int nz, int nx,
                       bool to_staging) {
  for (int f = 0; f < nf; ++f)
    for (int l = 0; l < ny; ++l)
      for (int k = 0; k < nz; ++k) {
        const size_t st = (((size_t)f * ny + l) * nz + k) * nx;   // staging row (y, z)
        const size_t ab = (((size_t)f * nz + k) * ny + l) * nx;   // ABI row (z, y)
        if (to_staging) std::memcpy(dst + st, src + ab, nx * sizeof(double));
        else std::memcpy(dst + ab, src + st, nx * sizeof(double));
      }
}

int ptt_set_state(ptt_ctx* c, int32_t member, const double* h) {
  if (!member_ok(c, member) || !h) return PTT_EINVAL;
  const ptt_params& p = c->prm[member];
  if (p.nz > 1) {
    std::vector<double> t((size_t)9 * p.ny * p.nz * p.nx);
    reorder_zy(h, t.data(), 9, p.ny, p.nz, p.nx, true);
    return upload_phys(c, member, t.data());
  }
  return upload_phys(c, member, h);
}

int ptt_get_state(ptt_ctx* c, int32_t member, double* h) {
  if (!member_ok(c, member) || !h) return PTT_EINVAL;
  auto [gi, b] = c->where[member];
  Group& g = c->groups[gi];
  const bool d3 = g.d.nz > 1;
  const size_t n = (size_t)(d3 ? 9 : 5) * g.d.N * g.d.nz * g.d.nx;
  CK(d3 ? launch_state_to_phys3(g.d, b, c->stream) : launch_state_to_phys(g.d, b, c->stream));
  if (d3) {
    std::vector<double> t(n);
    CK(cudaMemcpyAsync(t.data(), g.d.stage, n * 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    reorder_zy(t.data(), h, 9, g.d.N, g.d.nz, g.d.nx, false);
    return PTT_OK;
  }
  CK(cudaMemcpyAsync(h, g.d.stage, n * 8, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return PTT_OK;
}

int ptt_set_spectral(ptt_ctx* c, int32_t member, const double* h) {
  if (!member_ok(c, member) || !h) return PTT_EINVAL;
  auto [gi, b] = c->where[member];
  Group& g = c->groups[gi];
  const bool d3 = g.d.nz > 1;
  const int nf = d3 ? 9 : 5;
  const size_t NK = (size_t)g.d.N * g.d.KZ;
  CK(cudaMemcpyAsync(g.d.stageS, h, nf * NK * 16, cudaMemcpyHostToDevice, c->stream));
  CK(launch_transpose(g.d.stageS, g.d.X + (size_t)b * nf * NK, nf, g.d.N, g.d.KZ, c->stream));
  CK(d3 ? launch_reset_member3(g.d, b, c->stream) : launch_reset_member(g.d, b, c->stream));
  CK(d3 ? launch_diag3(g.d, c->stream, nullptr) : launch_diag(g.d, c->stream, nullptr));
  CK(cudaStreamSynchronize(c->stream));
  c->last_read[member] = -1;
  return PTT_OK;
}

int ptt_get_spectral(ptt_ctx* c, int32_t member, double* h) {
  if (!member_ok(c, member) || !h) return PTT_EINVAL;
  auto [gi, b] = c->where[member];
  Group& g = c->groups[gi];
  const int nf = (g.d.nz > 1) ? 9 : 5;
  const size_t NK = (size_t)g.d.N * g.d.KZ;
  CK(launch_transpose(g.d.X + (size_t)b * nf * NK, g.d.stageS, nf, g.d.KZ, g.d.N, c->stream));
  CK(cudaMemcpyAsync(h, g.d.stageS, nf * NK * 16, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return PTT_OK;
}

int ptt_explicit_rhs(ptt_ctx* c, int32_t member, double* h) {
  if (!member_ok(c, member) || !h) return PTT_EINVAL;
  auto [gi, b] = c->where[member];
  Group& g = c->groups[gi];
  const bool d3 = g.d.nz > 1;
  const int nf = d3 ? 9 : 5, nc = d3 ? 6 : 3;
  const size_t NK = (size_t)g.d.N * g.d.KZ;
  CK(d3 ? launch_explicit3(g.d, c->stream) : launch_explicit(g.d, c->stream));
  CK(launch_transpose(g.d.NR + (size_t)b * nf * NK, g.d.stageS, nc, g.d.KZ, g.d.N, c->stream));
  CK(launch_transpose(g.d.Rb + (size_t)b * 4 * NK, g.d.stageS + nc * NK, nf - nc, g.d.KZ, g.d.N,
                      c->stream));
  CK(cudaMemcpyAsync(h, g.d.stageS, nf * NK * 16, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return PTT_OK;
}

int ptt_step(ptt_ctx* c, int32_t nsteps) {
  if (!c || nsteps < 0) return PTT_EINVAL;
  if (nsteps == 0) return PTT_OK;
  CK(cudaGraphLaunch(c->exec[0], c->stream));
  for (int i = 1; i < nsteps; ++i) CK(cudaGraphLaunch(c->exec[1], c->stream));
  CK(cudaGraphLaunch(c->exec[2], c->stream));
  return PTT_OK;
}

// Poll the context stream until its work is done or `seconds` of wall-clock
// time have passed (seconds < 0: no limit): spin for the first 0.2 ms, then
// sleep in steps of at most 0.1 ms between queries.
static int wait_stream(ptt_ctx* c, double seconds) {
  const auto t0 = std::chrono::steady_clock::now();
  for (int it = 0;; ++it) {
    const cudaError_t e = cudaStreamQuery(c->stream);
    if (e == cudaSuccess) return PTT_OK;
    if (e != cudaErrorNotReady) return fail_cuda(e, "cudaStreamQuery", __LINE__);
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (seconds >= 0.0 && el >= seconds) {
      std::snprintf(g_last_error, sizeof(g_last_error),
                    "ptt_synchronize: work still in flight after %.3f s", el);
      return PTT_TIMEOUT;
    }
    if (el > 2e-4) std::this_thread::sleep_for(std::chrono::microseconds(el > 1e-3 ? 100 : 20));
  }
}

int ptt_set_timeout(ptt_ctx* c, double seconds) {
  if (!c || seconds != seconds) return PTT_EINVAL;
  c->timeout_s = seconds;
  return PTT_OK;
}

int ptt_synchronize_for(ptt_ctx* c, double seconds) {
  if (!c || seconds != seconds) return PTT_EINVAL;
  const int w = wait_stream(c, seconds);
  if (w) return w;
  int blown = 0;
  for (Group& g : c->groups) {
    std::vector<int> st(g.d.nb);
    CK(cudaMemcpy(st.data(), g.d.status, g.d.nb * sizeof(int), cudaMemcpyDeviceToHost));
    for (int v : st) blown |= (v != 0);
  }
  return blown ? PTT_BLOWUP : PTT_OK;
}

int ptt_synchronize(ptt_ctx* c) {
  if (!c) return PTT_EINVAL;
  return ptt_synchronize_for(c, c->timeout_s > 0.0 ? c->timeout_s : -1.0);
}

int ptt_diagnostics(ptt_ctx* c, int32_t member, ptt_diag* out, int32_t maxr, int32_t* nw) {
  if (!member_ok(c, member) || !out || maxr < 0 || !nw) return PTT_EINVAL;
  *nw = 0;
  auto [gi, b] = c->where[member];
  Group& g = c->groups[gi];
  long long cnt = 0;
  CK(cudaMemcpyAsync(&cnt, g.d.count + b, sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  long long first = c->last_read[member] + 1;
  if (first < cnt - kRing + 1) first = cnt - kRing + 1;
  if (first < 0) first = 0;
  const long long avail = cnt - first + 1;
  const int n = (int)(avail < maxr ? (avail > 0 ? avail : 0) : maxr);
  // records first .. first + n - 1 sit in ring slots s mod kRing: at most two
  // contiguous pieces
  const ptt_diag* ring = g.d.ring + (size_t)b * kRing;
  const int s0 = (int)(first % kRing);
  const int n1 = std::min(n, kRing - s0);
  if (n1 > 0)
    CK(cudaMemcpyAsync(out, ring + s0, (size_t)n1 * sizeof(ptt_diag), cudaMemcpyDeviceToHost, c->stream));
  if (n > n1)
    CK(cudaMemcpyAsync(out + n1, ring, (size_t)(n - n1) * sizeof(ptt_diag), cudaMemcpyDeviceToHost,
                       c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (n > 0) c->last_read[member] = first + n - 1;
  *nw = n;
  return PTT_OK;
}

int ptt_resample(ptt_ctx* dst, int32_t dm, ptt_ctx* src, int32_t sm) {
  if (!member_ok(dst, dm) || !member_ok(src, sm)) return PTT_EINVAL;
  if (dst->device != src->device) return PTT_EINVAL;
  auto [dgi, db] = dst->where[dm];
  auto [sgi, sb] = src->where[sm];
  const GroupDev& dg = dst->groups[dgi].d;
  const GroupDev& sg = src->groups[sgi].d;
  if ((dg.nz > 1) != (sg.nz > 1)) return PTT_EINVAL;
  if (dst == src && dm == sm) return PTT_OK;
  CK(cudaStreamSynchronize(src->stream));
  CK(launch_resample(dg, db, sg, sb, dst->stream));
  const bool d3 = dg.nz > 1;
  CK(d3 ? launch_reset_member3(dg, db, dst->stream) : launch_reset_member(dg, db, dst->stream));
  CK(d3 ? launch_diag3(dg, dst->stream, nullptr) : launch_diag(dg, dst->stream, nullptr));
  CK(cudaStreamSynchronize(dst->stream));
  dst->last_read[dm] = -1;
  return PTT_OK;
}

// Device milliseconds of `reps` launches of stages s0..s1 of one group.
// Time stages s0..s1 of one group (s0 < 0: only the diagnostics' two y
// transforms, which write scratch only).
static int time_stages_of(ptt_ctx* c, const GroupDev& d, int s0, int s1, int reps, float* ms) {
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  auto run = [&]() -> cudaError_t {
    if (s0 < 0) return (d.nz > 1) ? launch_diag_transforms3(d, c->stream) : launch_diag_transforms(d, c->stream);
    for (int s = s0; s <= s1; ++s) {
      cudaError_t e = (d.nz > 1) ? launch_stage3(d, s, c->stream, nullptr) : launch_stage(d, s, c->stream, nullptr);
      if (e) return e;
    }
    return cudaSuccess;
  };
  cudaError_t e = run();                       // warm-up
  if (!e) e = run();
  if (!e) e = cudaEventRecord(e0, c->stream);
  for (int r = 0; r < reps && !e; ++r) e = run();
  if (!e) e = cudaEventRecord(e1, c->stream);
  if (!e) e = cudaEventSynchronize(e1);
  if (!e) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e) return fail_cuda(e, "autotune timing", __LINE__);
  return PTT_OK;
}

int ptt_autotune(ptt_ctx* c, int32_t* choices, int32_t max_groups) {
  if (!c) return PTT_EINVAL;
  int optin = 0;
  CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
  CK(cudaStreamSynchronize(c->stream));
  const int reps = 4;
  for (size_t gi = 0; gi < c->groups.size(); ++gi) {
    GroupDev& d = c->groups[gi].d;
    const bool d3 = d.nz > 1;
    // threads per block of the fused x pass (stage 1); the in-place 3D
    // form runs 512
    if (!(d3 && xfused3_inplace(d.Mx, d.f32))) {
      int best = d.xthreads;
      float bt = 1e30f;
      for (int t = 128; t <= 512; t += 64) {
        d.xthreads = t;
        float ms = 0;
        int s = time_stages_of(c, d, 1, 1, reps, &ms);
        if (s) return s;
        if (ms < bt) { bt = ms; best = t; }
      }
      d.xthreads = best;
    }
    // columns per block of the y passes, then (3D) lines per block of the
    // z passes (stages 0 and 2)
    {
      const int cand[] = {1, 2, 4, 6, 8, 12, 16};
      int best = d.Ccol;
      float bt = 1e30f;
      for (int C : cand) {
        if (smem_ycols(C, d.M, d.f32) > (size_t)optin) continue;
        d.Ccol = C;
        float ms = 0;
        int s = time_stages_of(c, d, 0, 2, reps, &ms);
        if (s) return s;
        if (ms < bt) { bt = ms; best = C; }
      }
      d.Ccol = best;
    }
    // columns per block of the diagnostics' y transforms (energy grid, then
    // unpadded grid); only those two launches run, so records and
    // histograms are untouched
    for (int which = 0; which < 2; ++which) {
      const int cand[] = {1, 2, 4, 6, 8, 12, 16};
      int& cc = which == 0 ? d.CcolE : d.CcolU;
      const int P = which == 0 ? d.Me : d.Pu;
      int best = cc;
      float bt = 1e30f;
      for (int C : cand) {
        if (smem_ycols(C, P, 0) > (size_t)optin) continue;
        cc = C;
        float ms = 0;
        int s = time_stages_of(c, d, -1, -1, reps, &ms);
        if (s) return s;
        if (ms < bt) { bt = ms; best = C; }
      }
      cc = best;
    }
    if (d3) {
      // up to every x mode of a row in one block (whole 512-byte rows in and out)
      const int cand[] = {1, 2, 4, 8, 16, 32, 64};
      int best = d.zC;
      float bt = 1e30f;
      for (int C : cand) {
        if (C > d.K || smem_zcols3(C, d.Mz, d.f32) > (size_t)optin) continue;
        d.zC = C;
        float ms = 0;
        int s = time_stages_of(c, d, 0, 2, reps, &ms);
        if (s) return s;
        if (ms < bt) { bt = ms; best = C; }
      }
      d.zC = best;
    }
    if (choices && (int)gi < max_groups) {
      choices[3 * gi] = d.Ccol;
      choices[3 * gi + 1] = d3 ? d.zC : 0;
      choices[3 * gi + 2] = d.xthreads;
    }
  }
  return capture_step_graph(c);
}

int ptt_set_histograms(ptt_ctx* c, int32_t member, const double* lo, const double* hi) {
  if (!member_ok(c, member) || !lo || !hi) return PTT_EINVAL;
  auto [gi, b] = c->where[member];
  Group& g = c->groups[gi];
  double r[16];
  for (int q = 0; q < 8; ++q) {
    r[2 * q] = lo[q];
    r[2 * q + 1] = hi[q];
  }
  const size_t nh = (size_t)8 * (PTT_HIST_BINS + 2);
  CK(cudaMemcpyAsync(const_cast<double*>(g.d.hrange) + (size_t)b * 16, r, sizeof(r),
                     cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemsetAsync(g.d.hist + (size_t)b * nh, 0, nh * sizeof(unsigned long long), c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return PTT_OK;
}

int ptt_get_histograms(ptt_ctx* c, int32_t member, int64_t* counts) {
  if (!member_ok(c, member) || !counts) return PTT_EINVAL;
  auto [gi, b] = c->where[member];
  Group& g = c->groups[gi];
  const size_t nh = (size_t)8 * (PTT_HIST_BINS + 2);
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(counts, g.d.hist + (size_t)b * nh, nh * sizeof(int64_t), cudaMemcpyDeviceToHost));
  return PTT_OK;
}

int ptt_reset_moments(ptt_ctx* c, int32_t member) {
  if (!member_ok(c, member)) return PTT_EINVAL;
  auto [gi, b] = c->where[member];
  Group& g = c->groups[gi];
  CK(cudaMemsetAsync(g.d.macc + (size_t)b * kMacc, 0, kMacc * sizeof(double), c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return PTT_OK;
}

int ptt_midplane_moments(ptt_ctx* c, int32_t member, double* moments, int64_t* nrecords) {
  if (!member_ok(c, member) || !moments) return PTT_EINVAL;
  auto [gi, b] = c->where[member];
  Group& g = c->groups[gi];
  double out[kMacc];
  CK(launch_window_moments(g.d, b, (double)g.d.nx * g.d.nz, c->stream));
  CK(cudaMemcpyAsync(out, g.d.statout, sizeof(out), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (int i = 0; i < 32; ++i) moments[i] = out[i];
  if (nrecords) *nrecords = (int64_t)out[32];
  return PTT_OK;
}

int ptt_histogram_l1(ptt_ctx* a, int32_t member_a, ptt_ctx* b, int32_t member_b, double* l1) {
  if (!member_ok(a, member_a) || !member_ok(b, member_b) || !l1) return PTT_EINVAL;
  auto [ga, ia] = a->where[member_a];
  auto [gb, ib] = b->where[member_b];
  const size_t nh = (size_t)8 * (PTT_HIST_BINS + 2);
  const GroupDev& da = a->groups[ga].d;
  const GroupDev& db = b->groups[gb].d;
  double out[8];
  if (b != a) CK(cudaStreamSynchronize(b->stream));
  CK(launch_hist_l1(da.hist + (size_t)ia * nh, db.hist + (size_t)ib * nh, da.statout, a->stream));
  CK(cudaMemcpyAsync(out, da.statout, sizeof(out), cudaMemcpyDeviceToHost, a->stream));
  CK(cudaStreamSynchronize(a->stream));
  for (int q = 0; q < 8; ++q) l1[q] = out[q];
  return PTT_OK;
}

static size_t ckpt_bytes(const Group& g) {
  const size_t NK = (size_t)g.d.N * g.d.KZ;
  const size_t nf = (g.d.nz > 1) ? 9 : 5, ne = (g.d.nz > 1) ? 8 : 4;
  return 64 + (nf + 8 * ne) * NK * 16;
}

int ptt_checkpoint_size(ptt_ctx* c, int32_t member, size_t* bytes) {
  if (!member_ok(c, member) || !bytes) return PTT_EINVAL;
  *bytes = ckpt_bytes(c->groups[c->where[member].first]);
  return PTT_OK;
}

// Checkpoint copies: one cudaMemcpyAsync per array on the context stream
// (ordered after the steps already launched), then one synchronisation, so
// the calls return with the copies done, as their contract states.
int ptt_get_checkpoint(ptt_ctx* c, int32_t member, void* h, size_t bytes) {
  if (!member_ok(c, member) || !h) return PTT_EINVAL;
  auto [gi, b] = c->where[member];
  Group& g = c->groups[gi];
  if (bytes < ckpt_bytes(g)) return PTT_EINVAL;
  const size_t NK = (size_t)g.d.N * g.d.KZ, nb = g.d.nb;
  const size_t nf = (g.d.nz > 1) ? 9 : 5, ne = (g.d.nz > 1) ? 8 : 4;
  char* p = (char*)h;
  long long cnt = 0;
  int st = 0;
  cudaStream_t s = c->stream;
  CK(cudaMemcpyAsync(&cnt, g.d.count + b, 8, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&st, g.d.status + b, 4, cudaMemcpyDeviceToHost, s));
  char* q = p + 64;
  CK(cudaMemcpyAsync(q, g.d.X + b * nf * NK, nf * NK * 16, cudaMemcpyDeviceToHost, s));
  q += nf * NK * 16;
  for (int k = 0; k < 4; ++k) {
    CK(cudaMemcpyAsync(q, g.d.Eh + ((size_t)k * nb + b) * ne * NK, ne * NK * 16, cudaMemcpyDeviceToHost, s));
    q += ne * NK * 16;
    CK(cudaMemcpyAsync(q, g.d.Nh + ((size_t)k * nb + b) * ne * NK, ne * NK * 16, cudaMemcpyDeviceToHost, s));
    q += ne * NK * 16;
  }
  CK(cudaStreamSynchronize(s));
  int64_t hdr[8] = {0x70747463, g.d.nx, g.d.N, cnt, st, g.d.nz, 0, 0};
  std::memcpy(p, hdr, 64);
  return PTT_OK;
}

int ptt_set_checkpoint(ptt_ctx* c, int32_t member, const void* h, size_t bytes) {
  if (!member_ok(c, member) || !h) return PTT_EINVAL;
  auto [gi, b] = c->where[member];
  Group& g = c->groups[gi];
  if (bytes < ckpt_bytes(g)) return PTT_EINVAL;
  const size_t NK = (size_t)g.d.N * g.d.KZ, nb = g.d.nb;
  const size_t nf = (g.d.nz > 1) ? 9 : 5, ne = (g.d.nz > 1) ? 8 : 4;
  const char* p = (const char*)h;
  int64_t hdr[8];
  std::memcpy(hdr, p, 64);
  if (hdr[0] != 0x70747463 || hdr[1] != g.d.nx || hdr[2] != g.d.N || hdr[5] != g.d.nz) return PTT_EINVAL;
  p += 64;
  const long long cnt = hdr[3];
  const int st = (int)hdr[4];
  cudaStream_t s = c->stream;
  CK(cudaMemcpyAsync(g.d.count + b, &cnt, 8, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(g.d.status + b, &st, 4, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(g.d.X + b * nf * NK, p, nf * NK * 16, cudaMemcpyHostToDevice, s));
  p += nf * NK * 16;
  for (int k = 0; k < 4; ++k) {
    CK(cudaMemcpyAsync(g.d.Eh + ((size_t)k * nb + b) * ne * NK, p, ne * NK * 16, cudaMemcpyHostToDevice, s));
    p += ne * NK * 16;
    CK(cudaMemcpyAsync(g.d.Nh + ((size_t)k * nb + b) * ne * NK, p, ne * NK * 16, cudaMemcpyHostToDevice, s));
    p += ne * NK * 16;
  }
  // the sources (cnt, st on this stack frame; the caller's buffer) must stay
  // valid until the copies have run
  CK(cudaStreamSynchronize(s));
  c->last_read[member] = cnt;
  return PTT_OK;
}

int ptt_time_stages(ptt_ctx* c, int32_t nsteps, double* ms) {
  if (!c || nsteps < 0 || !ms) return PTT_EINVAL;
  const int G = (int)c->groups.size();
  std::vector<cudaEvent_t> ev((size_t)G * (PTT_NSTAGES + 1), nullptr);
  for (auto& e : ev) CK(cudaEventCreate(&e));
  int rc = PTT_OK;
  for (int st = 0; st < nsteps && rc == PTT_OK; ++st) {
    for (int gi = 0; gi < G; ++gi) {
      cudaEvent_t* E = &ev[(size_t)gi * (PTT_NSTAGES + 1)];
      cudaError_t e = cudaEventRecord(E[0], c->stream);
      for (int s = 0; s < PTT_NSTAGES && !e; ++s) {
        const GroupDev& gd = c->groups[gi].d;
        e = (gd.nz > 1) ? launch_stage3(gd, s, c->stream, nullptr) : launch_stage(gd, s, c->stream, nullptr);
        if (!e) e = cudaEventRecord(E[s + 1], c->stream);
      }
      if (e) { rc = fail_cuda(e, "ptt_time_stages launch", __LINE__); break; }
    }
    if (rc) break;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e) { rc = fail_cuda(e, "ptt_time_stages sync", __LINE__); break; }
    for (int gi = 0; gi < G; ++gi) {
      cudaEvent_t* E = &ev[(size_t)gi * (PTT_NSTAGES + 1)];
      for (int s = 0; s < PTT_NSTAGES; ++s) {
        float t = 0.f;
        cudaEventElapsedTime(&t, E[s], E[s + 1]);
        ms[s] += t;
      }
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  return rc;
}

int ptt_stage_work(ptt_ctx* c, double* flops, double* bytes, int32_t* launches) {
  if (!c || !flops || !bytes || !launches) return PTT_EINVAL;
  auto fft = [](double n) { return 5.0 * n * std::log2(n); };
  const int nlaunch[PTT_NSTAGES] = {1, 1, 1, 2, 7};
  for (int s = 0; s < PTT_NSTAGES; ++s) { flops[s] = 0.0; bytes[s] = 0.0; launches[s] = 0; }
  for (Group& g : c->groups) {
    const GroupDev& d = g.d;
    if (d.nz > 1) {   // 3D
      const double nb = d.nb, K = d.K, KZ = d.KZ, N = d.N, NK = N * KZ, M = d.M, Mz = d.Mz, Je = d.Me;
      const double z = 16.0;
      flops[0] += nb * (17.0 * KZ * (fft(M) + 8.0 * M) + 8.0 * KZ * N * 4.0 + 26.0 * M * K * fft(Mz));
      bytes[0] += nb * z * (9.0 * NK + 26.0 * M * Mz * K);
      flops[1] += nb * M * Mz * (23.0 * fft(d.Mx) + 200.0 * d.Mx);
      bytes[1] += nb * z * (26.0 + 9.0) * M * Mz * K;
      flops[2] += nb * (9.0 * M * K * fft(Mz) + 9.0 * KZ * (fft(M) + 8.0 * M));
      bytes[2] += nb * z * (9.0 * M * Mz * K + 9.0 * NK);
      flops[3] += nb * NK * (8.0 * 4.0 + 8.0 * 4.0 * 8.0 + 16.0 * 24.0 / 2.0);
      bytes[3] += nb * (z * NK * (9.0 + 9.0 + 64.0 + 16.0 + 9.0) + 8.0 * NK * 10.0);
      flops[4] += nb * (KZ * fft(d.Pu) + N * K * fft(d.nz) + N * d.nz * fft(d.nx) +
                        3.0 * KZ * (fft(Je) + 8.0 * Je) + 8.0 * Je * KZ * 3.0);
      bytes[4] += nb * (z * (9.0 * NK + 3.0 * 2.0 * Je * KZ) + 8.0 * 2.0 * N * d.nz * d.nx);
      const int nl3[PTT_NSTAGES] = {2, 1, 2, 2, 10};
      for (int s = 0; s < PTT_NSTAGES; ++s) launches[s] += nl3[s];
      continue;
    }
    const double nb = d.nb, K = d.K, N = d.N, NK = N * K, rows = d.M, Je = d.Me;
    const double z = 16.0, r = 8.0;  // bytes of a complex / real double
    // 0: 9 complex columns, DCT-III on the M Gauss points (one FFT of M) + 4 d/dy
    flops[0] += nb * (9.0 * K * (fft(d.M) + 8.0 * d.M) + 4.0 * K * N * 4.0);
    bytes[0] += nb * z * (5.0 * NK + 9.0 * rows * K);
    // 1: per padded row 7 inverse + 3 forward complex FFTs of Mx, 42 flops of products per point
    flops[1] += nb * rows * (10.0 * fft(d.Mx) + 42.0 * d.Mx);
    bytes[1] += nb * z * (9.0 + 5.0) * rows * K;
    // 2: 5 complex columns, DCT-II
    flops[2] += nb * 5.0 * K * (fft(d.M) + 8.0 * d.M);
    bytes[2] += nb * z * (5.0 * rows * K + 5.0 * NK);
    // 3: 6 recurrences, SBDF sums over 4 levels of 8 fields, 8 tau sweeps
    flops[3] += nb * NK * (6.0 * 4.0 + 4.0 * 4.0 * 8.0 + 8.0 * 24.0 / 2.0);
    bytes[3] += nb * (z * NK * (5.0 + 5.0 + 32.0 + 8.0 + 5.0) + r * NK * 10.0);
    // 4: diagnostics: DCT-I of one field (FFT of 2(N-1)), DCT-III of u, v on Me points,
    //    x transforms of the unpadded rows and the mid-plane, reductions
    flops[4] += nb * (K * fft(d.Pu) + 2.0 * K * (fft(d.Me) + 8.0 * d.Me) + N * fft(d.nx) +
                      3.0 * fft(d.nx) + NK * 10.0 + 8.0 * Je * K);
    bytes[4] += nb * (z * (5.0 * NK + 2.0 * 2.0 * Je * K + 2.0 * NK) + r * 2.0 * N * d.nx);
    for (int s = 0; s < PTT_NSTAGES; ++s) launches[s] += nlaunch[s];
  }
  return PTT_OK;
}

int ptt_set_launch_mode(ptt_ctx* c, int32_t mode) {
  if (!c || (mode != 0 && mode != 1)) return PTT_EINVAL;
  if (mode == 1 && !c->multi_dev) return PTT_ENOTSUP;
  CK(cudaStreamSynchronize(c->stream));
  c->launch_mode = mode;
  return capture_step_graph(c);
}

int ptt_launches_per_step(ptt_ctx* c, int32_t* n) {
  if (!c || !n) return PTT_EINVAL;
  *n = c->launches;
  return PTT_OK;
}

int ptt_destroy(ptt_ctx* c) {
  if (!c) return PTT_EINVAL;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  for (int k = 0; k < 3; ++k) {
    if (c->exec[k]) cudaGraphExecDestroy(c->exec[k]);
    if (c->graph[k]) cudaGraphDestroy(c->graph[k]);
  }
  if (c->cap) cudaStreamDestroy(c->cap);
  for (auto s2 : c->gstreams) if (s2) cudaStreamDestroy(s2);
  for (auto s2 : c->dstreams) if (s2) cudaStreamDestroy(s2);
  for (auto s2 : c->pstreams) if (s2) cudaStreamDestroy(s2);
  for (auto e2 : c->gevents) if (e2) cudaEventDestroy(e2);
  for (auto e2 : c->devents) if (e2) cudaEventDestroy(e2);
  for (auto e2 : c->pevents) if (e2) cudaEventDestroy(e2);
  if (c->multi) multi2d_destroy(c->multi);
  delete c;
  return PTT_OK;
}

const char* ptt_last_error(void) { return g_last_error; }

const char* ptt_status_string(int s) {
  switch (s) {
    case PTT_OK: return "ok";
    case PTT_BLOWUP: return "blow-up detected";
    case PTT_EINVAL: return "invalid argument";
    case PTT_ENOMEM: return "workspace too small";
    case PTT_ECUDA: return "CUDA runtime error";
    case PTT_TIMEOUT: return "bounded wait expired";
    case PTT_ENOTSUP: return "not supported by this library";
    default: return "unknown status";
  }
}

}  // extern "C"
