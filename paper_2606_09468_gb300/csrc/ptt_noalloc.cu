// Workspace-free variant of the explicit right-hand side (ptt_explicit_rhs_noalloc).
//
// Some callers cannot allocate device memory: code that runs inside a host
// library with a fixed memory budget handed out by someone else, plugins
// whose device memory is owned by the embedding application, or real-time
// loops in which an allocation (and the implicit synchronisation it brings)
// is not allowed.  For them the padded-grid intermediates of this entry
// point live in one file-scope device array, g_noalloc_scratch, sized
// kNoAllocBytes.  The array is part of the library's device image: every GPU
// on which the library is loaded holds those bytes until the process exits.
//
// In host code the name g_noalloc_scratch is a host-side stand-in, not a
// device address; the device address is looked up with cudaGetSymbolAddress
// on every call (with the caller's device current) and passed to the kernels.
#include <cstdio>
#include <mutex>
#include <vector>

#include "ptt_internal.h"

namespace {

constexpr size_t kNoAllocBytes = size_t(48) << 20;  // 48 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_mu;
void* g_dev_ptr[kMaxDevices] = {};   // address the kernels' attributes were last set for

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Device address of the scratch array on the current device, looked up on
// every call (cudaGetSymbolAddress allocates nothing), so that a device reset
// or another context on the same ordinal never leaves a stale address
// behind.  Whenever the address differs from the one seen before on this
// ordinal, the kernels' dynamic shared-memory limit is raised again.
int scratch_for_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e) {
    ptt::set_last_error(cudaGetErrorString(e));
    return PTT_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return PTT_EINVAL;
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    char msg[256];
    std::snprintf(msg, sizeof(msg), "cudaGetSymbolAddress(g_noalloc_scratch): %s",
                  cudaGetErrorString(e));
    ptt::set_last_error(msg);
    return PTT_ECUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_dev_ptr[dev] != p) {
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (!e) e = ptt::set_kernel_attributes(optin);
    if (e) {
      ptt::set_last_error(cudaGetErrorString(e));
      return PTT_ECUDA;
    }
    g_dev_ptr[dev] = p;
  }
  *out = p;
  return PTT_OK;
}

}  // namespace

extern "C" int ptt_explicit_rhs_noalloc(const ptt_params* p, const double* d_spec, double* d_out,
                                        void* cuda_stream) {
  if (!p || !d_spec || !d_out) return PTT_EINVAL;
  if (((uintptr_t)d_spec & 15) || ((uintptr_t)d_out & 15) || d_spec == d_out) return PTT_EINVAL;
  ptt::GroupDev g{};
  ptt::MemberPrm prm{};
  std::vector<double2> twP, twMx, tw4;
  std::vector<double> tt[2];
  std::vector<int> tk[2];
  int s = ptt::shape_plan(*p, g, twP, twMx, tw4, prm, tt, tk);
  if (s) return s;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  {
    // the host-to-device copies and the final synchronisation below are not
    // allowed while the stream is being captured
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) {
      char msg[256];
      std::snprintf(msg, sizeof(msg), "ptt_explicit_rhs_noalloc: cudaStreamIsCapturing: %s",
                    cudaGetErrorString(e));
      ptt::set_last_error(msg);
      return PTT_ECUDA;
    }
    if (cs != cudaStreamCaptureStatusNone) {
      ptt::set_last_error("ptt_explicit_rhs_noalloc: the stream is being captured");
      return PTT_EINVAL;
    }
  }
  const size_t rows = (size_t)g.M, K = g.K, NK = (size_t)g.N * K;
  // layout of the scratch array
  size_t off = 0;
  const size_t oX = off; off = align256(off + 5 * NK * sizeof(double2));
  const size_t oNR = off; off = align256(off + 5 * NK * sizeof(double2));
  const size_t oRb = off; off = align256(off + 2 * NK * sizeof(double2));
  const size_t oYp = off; off = align256(off + 9 * rows * K * sizeof(double2));
  const size_t oZp = off; off = align256(off + 5 * rows * K * sizeof(double2));
  const size_t oTP = off; off = align256(off + twP.size() * sizeof(double2));
  const size_t oTM = off; off = align256(off + twMx.size() * sizeof(double2));
  const size_t oT4 = off; off = align256(off + tw4.size() * sizeof(double2));
  size_t oTT[2], oTK[2];
  for (int i = 0; i < 2; ++i) {
    oTT[i] = off; off = align256(off + tt[i].size() * sizeof(double));
    oTK[i] = off; off = align256(off + tk[i].size() * sizeof(int));
  }
  const size_t oPr = off; off = align256(off + sizeof(ptt::MemberPrm));
  const size_t oSt = off; off = align256(off + sizeof(int));
  const size_t oCn = off; off = align256(off + sizeof(long long));
  if (off > kNoAllocBytes) {
    char msg[256];
    std::snprintf(msg, sizeof(msg),
                  "ptt_explicit_rhs_noalloc: nx=%d ny=%d needs %zu bytes of scratch, the "
                  "static array holds %zu",
                  p->nx, p->ny, off, kNoAllocBytes);
    ptt::set_last_error(msg);
    return PTT_ENOMEM;
  }
  void* base = nullptr;
  s = scratch_for_current_device(&base);
  if (s) return s;
  char* b = (char*)base;
  g.X = (double2*)(b + oX);     // input in the kernels' mode-major layout
  g.NR = (double2*)(b + oNR);   // N_cxx, N_cxy, N_cyy, N_u, N_v
  g.Rb = (double2*)(b + oRb);   // H_x, H_y
  g.Yp = (double2*)(b + oYp);
  g.Zp = (double2*)(b + oZp);
  g.plP.tw = (const double2*)(b + oTP);
  g.plMx.tw = (const double2*)(b + oTM);
  ptt::FftPlan* pls[2] = {&g.plP, &g.plMx};
  for (int i = 0; i < 2; ++i) {
    pls[i]->tt = (const double*)(b + oTT[i]);
    pls[i]->tk = (const int*)(b + oTK[i]);
  }
  g.tw4P = (const double2*)(b + oT4);                      // forward table, M entries
  g.tw4Pi = (const double2*)(b + oT4) + tw4.size() / 2;    // inverse table, M entries
  g.prm = (ptt::MemberPrm*)(b + oPr);
  g.status = (int*)(b + oSt);
  g.count = (long long*)(b + oCn);
  cudaError_t e = cudaSuccess;
  // status and step counter must read zero; tables and parameters are
  // rewritten on every call (the array keeps the previous call's contents)
  e = cudaMemsetAsync(b + oSt, 0, sizeof(int), st);
  if (!e) e = cudaMemsetAsync(b + oCn, 0, sizeof(long long), st);
  if (!e) e = cudaMemcpyAsync(b + oTP, twP.data(), twP.size() * sizeof(double2),
                              cudaMemcpyHostToDevice, st);
  if (!e) e = cudaMemcpyAsync(b + oTM, twMx.data(), twMx.size() * sizeof(double2),
                              cudaMemcpyHostToDevice, st);
  if (!e) e = cudaMemcpyAsync(b + oT4, tw4.data(), tw4.size() * sizeof(double2),
                              cudaMemcpyHostToDevice, st);
  for (int i = 0; i < 2 && !e; ++i) {
    e = cudaMemcpyAsync(b + oTT[i], tt[i].data(), tt[i].size() * sizeof(double),
                        cudaMemcpyHostToDevice, st);
    if (!e) e = cudaMemcpyAsync(b + oTK[i], tk[i].data(), tk[i].size() * sizeof(int),
                                cudaMemcpyHostToDevice, st);
  }
  if (!e) e = cudaMemcpyAsync(b + oPr, &prm, sizeof(prm), cudaMemcpyHostToDevice, st);
  if (!e) e = ptt::launch_transpose((const double2*)d_spec, g.X, 5, g.N, g.K, st);
  if (!e) e = ptt::launch_explicit(g, st);
  if (!e) e = ptt::launch_transpose(g.NR, (double2*)d_out, 3, g.K, g.N, st);
  if (!e) e = ptt::launch_transpose(g.Rb, (double2*)d_out + 3 * NK, 2, g.K, g.N, st);
  // the host tables must outlive the copies above
  const cudaError_t es = cudaStreamSynchronize(st);
  if (!e) e = es;
  if (e) {
    char msg[256];
    std::snprintf(msg, sizeof(msg), "ptt_explicit_rhs_noalloc: %s", cudaGetErrorString(e));
    ptt::set_last_error(msg);
    return PTT_ECUDA;
  }
  return PTT_OK;
}
