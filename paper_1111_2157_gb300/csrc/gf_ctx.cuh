// Private to the C-ABI translation units of libgf (gf_api.cu, gf_api_pole.cu): the
// context behind the opaque gf_ctx of include/gf.h and the host helpers both use.
// Nothing here is part of the C-ABI.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <map>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gf.h"
#include "gf_internal.cuh"

using gf::Item;
using gf::KInfo;
using gf::SInfo;

namespace gf_host {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  template <class T>
  T* as() const { return static_cast<T*>(p); }
};

inline cudaError_t ensure(DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return cudaSuccess;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e == cudaSuccess) b.bytes = bytes;
  return e;
}

inline void release(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

// NVTX range around a C-ABI call (visible in Nsight timelines; no cost without a tool).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// A start/stop pair of timing events owned by one scope: destroyed on every return path.
struct ScopedEvents {
  cudaEvent_t start = nullptr, stop = nullptr;
  cudaError_t create() {
    const cudaError_t e = cudaEventCreate(&start);
    return e != cudaSuccess ? e : cudaEventCreate(&stop);
  }
  ScopedEvents() = default;
  ScopedEvents(const ScopedEvents&) = delete;
  ScopedEvents& operator=(const ScopedEvents&) = delete;
  ~ScopedEvents() {
    if (start) cudaEventDestroy(start);
    if (stop) cudaEventDestroy(stop);
  }
};

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int d) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != d) cudaSetDevice(d);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// Trigamma psi'(x) for x > 0: recurrence up to x >= 20, then the asymptotic series
// psi'(x) ~ 1/x + 1/(2x^2) + sum_k B_2k / x^(2k+1).
}  // namespace gf_host

using namespace gf_host;


// Window buckets: one launch per bucket, tiles sized to the bucket's largest window.
constexpr int kNumBuckets = 6;
constexpr int kBucketBounds[kNumBuckets] = {8, 16, 40, 64, 96, 1 << 30};
inline int gf_bucket(int nb) {
  for (int i = 0; i < kNumBuckets - 1; ++i)
    if (nb <= kBucketBounds[i]) return i;
  return kNumBuckets - 1;
}

struct gf_ctx {
  int n_sys = 0, n_k = 0, n_iw = 0, precision = 0, in_dtype = 0, tail_order = 2, device = 0;
  // input dtype of each system's blocks (gf_desc.system_dtype, else in_dtype for all), and the
  // first complex element of each system in the packed H, diagonal-H, P, Sigma and Sigma_inf
  // arrays ([n_sys + 1], last = total)
  std::vector<int> sys_dtype;
  std::vector<int64_t> sysH, sysD, sysP, sysSig, sysSinf;
  cudaStream_t stream = nullptr;
  std::vector<int> nb, ksys, msys;
  std::vector<double> beta, wk;
  std::vector<KInfo> kinfo;
  std::vector<SInfo> sinfo;
  std::vector<int64_t> offD;  // prefix sums of nb (diagonal H input)
  int64_t totH = 0, totP = 0, totSig = 0, totSinf = 0, totNb = 0;
  int nbmax = 0, mmax = 0;
  int sm_count = 0, smem_optin = 0;
  int chunk_w = 1, n_chunks = 1;
  size_t gq_budget = 0;
  // work items: the k-group list of the k-reductions, batch after batch (groups
  // [batch_g0[b], batch_g0[b+1]) from item batch_item0[b]), sorted by decreasing window in
  // each batch; then the single-k list of the other modes from all_item0
  std::vector<Item> items;
  std::vector<int> batch_g0, batch_item0;
  int n_items_all = 0, all_item0 = 0;
  int kg = 1, n_groups = 0;                // k-points per group, number of groups
  std::vector<int> kperm, group_k0, group_nk;  // group g: kperm[group_k0[g] .. + group_nk[g])
  std::vector<int> sys_g0, sys_g1;         // groups of system s: [sys_g0[s], sys_g1[s])
  DevBuf kperm_d, sysg_d;  // kperm, then sys_g0 | sys_g1
  DevBuf H, P, Sig, Sinf, Einf, trHE, kinfo_d, sinfo_d, items_d, offD_d, mu, nbar, gbar, status,
      queue, stage, occ_part, rho_part, rho_out, gq, kN, kdN, kNc, sysout, a_scratch, mubar_part,
      mubar_sys, gacc, sysout2;
  DevBuf Hd, Pd, Sd, Gbd;  // FP32-pair copies (GF_PREC_MIXED and GF_PREC_PAIR)
  DevBuf Hs, Ps, Ss;       // single-word FP32 copies (GF_PREC_MIXED)
  bool have_H = false, have_P = false, have_S = false, einf_dirty = true;
  bool have_gbar_for_call = false;
  // pinned host staging: mu [S] | n_bar [S] | status | outputs [2S] | mu_bar [S] | outputs [2S]
  double* hpin = nullptr;
  double* hp_mu() { return hpin; }
  double* hp_nbar() { return hpin + n_sys; }
  double* hp_status() { return hpin + 2 * n_sys; }
  double* hp_sys() { return hpin + 2 * n_sys + 1; }
  double* hp_mubar() { return hpin + 4 * n_sys + 1; }
  double* hp_sys2() { return hpin + 5 * n_sys + 1; }
  std::string err;
  std::map<int, int> tuned;  // candidate chosen by the autotuner, per (mode, bucket)
  int bucket_nbmax[kNumBuckets] = {0, 0, 0, 0, 0, 0};
  // CUDA-graph replay of the N(mu) evaluation (GF_FLAG_GRAPH)
  bool use_graph = false;
  int occ_calls = 0;
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t ev_user = nullptr;
  cudaGraphExec_t occ_exec = nullptr;
  bool capturing = false;
  int64_t occ_launches = 0, occ_points = 0;
  double occ_flops = 0.0;
  std::string tune_log;
  int64_t last_launches = 0, last_points = 0;
  double last_kernel_ms = 0.0, last_flops = 0.0;
  // CUDA event pairs around the point-kernel launches of the current call
  std::vector<cudaEvent_t> ev;
  int ev_used = 0;
  // low-rank (eigenbasis) algorithm, GF_FLAG_LOWRANK
  bool lowrank = false, lr_dirty = true;
  // set by gf_create once the device ordinal is known to be valid: from then on a failed
  // creation is undone by gf_destroy, before that by a plain delete (no CUDA call)
  bool device_checked = false;
  DevBuf lr_eps, lr_U, lr_Pt, lr_T, lr_ws;
  // DMFT step and projector construction
  DevBuf eimp, eimp_part, gl_in, delta, wraw, vdc;
  // pole form of Sigma (gf_set_sigma_poles) and the pseudo-Hamiltonian path
  bool have_poles = false;
  int64_t pole_v_elems = 0, pole_e_elems = 0;
  std::vector<gf::PInfo> pinfo;
  int nps_max = 0;
  DevBuf poles, Vp, Sinf_p, pinfo_d, eoff_d, phioff_d, eout, phiout, pole_ws, wbout, kHks, kEps,
      eps_grid, dos, pdos, pdos_off, pole_part, pole_vs, pole_es, voff_d, mu_prev;
};

namespace gf_host {

// Room for n timing events in c->ev, taken before an event is created so that the push_back
// which stores it cannot throw and leak it.
inline void reserve_events(gf_ctx* c, int n) {
  if (c->ev.capacity() < (size_t)n) c->ev.reserve(std::max<size_t>(2 * (size_t)n, 16));
}

inline gf_status fail(gf_ctx* c, gf_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

// Handler of the function-try-block around every entry point that runs host code able to
// throw (growth of std::vector and std::string, std::mutex), so that no C++ exception crosses
// the C ABI: a failed or oversized host allocation becomes GF_ENOMEM, anything else GF_EINVAL.
// The message goes to the context, or to gf_last_error(NULL) when there is none.
inline gf_status caught(const gf_ctx* c) noexcept {
  if (!c) return gf::caught_global();
  const char* msg = "";
  const gf_status s = gf::exception_status(&msg);
  try {
    const_cast<gf_ctx*>(c)->err = msg;
  } catch (...) {
  }
  return s;
}

#define GF_CU(call)                                                                        \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(c, e_ == cudaErrorMemoryAllocation ? GF_ENOMEM : GF_ECUDA,               \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                     \
  } while (0)

// Copy n complex numbers of one dtype from a host or device pointer into a complex128
// device array (complex64 upcast on the device).
inline gf_status load_complex_dtype(gf_ctx* c, const void* src, int64_t n, int dtype, double2* dst) {
  if (n <= 0) return GF_OK;
  if (dtype == GF_C128) {
    GF_CU(cudaMemcpyAsync(dst, src, (size_t)n * 16, cudaMemcpyDefault, c->stream));
  } else {
    GF_CU(ensure(c->stage, (size_t)n * 8));
    GF_CU(cudaMemcpyAsync(c->stage.p, src, (size_t)n * 8, cudaMemcpyDefault, c->stream));
    GF_CU(gf::launch_upcast(c->stage.as<float2>(), dst, n, c->stream));
  }
  return GF_OK;
}

// Copy a packed per-system input (system s holds complex elements [sysoff[s], sysoff[s+1]) of
// the destination, stored in the source in the dtype of system s, the systems' blocks one
// after the other) into a complex128 device array.  Consecutive systems of one dtype move
// in one copy.
inline gf_status load_complex(gf_ctx* c, const void* src, const std::vector<int64_t>& sysoff,
                              double2* dst) {
  const unsigned char* in = static_cast<const unsigned char*>(src);
  size_t byte = 0;
  for (int s0 = 0; s0 < c->n_sys;) {
    int s1 = s0 + 1;
    while (s1 < c->n_sys && c->sys_dtype[s1] == c->sys_dtype[s0]) ++s1;
    const int64_t e0 = sysoff[s0], n = sysoff[s1] - e0;
    const int dt = c->sys_dtype[s0];
    gf_status st = load_complex_dtype(c, in + byte, n, dt, dst + e0);
    if (st) return st;
    byte += (size_t)n * (dt == GF_C128 ? 16 : 8);
    // the staging buffer of a complex64 run is reused by the next run: wait for the upcast
    if (dt == GF_C64 && s1 < c->n_sys) GF_CU(cudaStreamSynchronize(c->stream));
    s0 = s1;
  }
  return GF_OK;
}

// FP32 copies of an uploaded input (n complex numbers in src): FP32 pairs for
// GF_PREC_MIXED and GF_PREC_PAIR, and single words for GF_PREC_MIXED.
inline gf_status derive_f32(gf_ctx* c, const DevBuf& src, DevBuf& pair, DevBuf* single, int64_t n) {
  if (c->precision == GF_PREC_FP64 || n <= 0) return GF_OK;
  GF_CU(gf::launch_split_df64(src.as<double2>(), pair.as<float4>(), n, c->stream));
  if (c->precision == GF_PREC_MIXED && single)
    GF_CU(gf::launch_round_f32(src.as<double2>(), single->as<float2>(), n, c->stream));
  return GF_OK;
}

inline gf_status sync_and_check(gf_ctx* c) {
  GF_CU(cudaMemcpyAsync(c->hp_status(), c->status.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  GF_CU(cudaStreamSynchronize(c->stream));
  for (int i = 0; i + 1 < c->ev_used; i += 2) {
    float ms = 0.f;
    GF_CU(cudaEventElapsedTime(&ms, c->ev[i], c->ev[i + 1]));
    c->last_kernel_ms += ms;
  }
  c->ev_used = 0;
  int flags = 0;
  std::memcpy(&flags, c->hp_status(), sizeof(int));
  if (flags & gf::kFlagSingular)
    return fail(c, GF_ESINGULAR, "zero or non-finite pivot in a (k, i w_n) inverse");
  if (flags & 2) return fail(c, GF_ENOTCONV, "Jacobi eigensolver did not converge in 40 sweeps");
  return GF_OK;
}

inline gf_status upload_mu(gf_ctx* c, const double* mu) {
  if (!mu) return fail(c, GF_EINVAL, "mu is NULL");
  for (int s = 0; s < c->n_sys; ++s) {
    if (!std::isfinite(mu[s])) return fail(c, GF_EINVAL, "mu is not finite");
    c->hp_mu()[s] = mu[s];
  }
  GF_CU(cudaMemcpyAsync(c->mu.p, c->hp_mu(), sizeof(double) * c->n_sys, cudaMemcpyHostToDevice,
                        c->stream));
  return GF_OK;
}

inline void reset_stats(gf_ctx* c) {
  c->last_launches = 0;
  c->last_points = 0;
  c->last_kernel_ms = 0.0;
  c->last_flops = 0.0;
  c->ev_used = 0;
}

// Safeguarded Newton search of mu with N(mu) = n_target per system (Eq. fix_mu):
// N is increasing in mu (dN/dmu > 0); a Newton step is capped at 4 eV while
// the bracket is one-sided and replaced by bisection when it leaves the
// bracket.  eval(mu, N, dN/dmu) evaluates all systems at once.
template <class Eval>
gf_status newton_mu(gf_ctx* c, const double* n_target, double tol, int32_t max_iter,
                    double* mu_inout, int32_t* iters_out, Eval eval) {
  if (!n_target || !mu_inout) return fail(c, GF_EINVAL, "n_target or mu_inout is NULL");
  if (!(tol > 0.0) || max_iter < 1) return fail(c, GF_EINVAL, "tol must be > 0 and max_iter >= 1");
  const int S = c->n_sys;
  const double inf = std::numeric_limits<double>::infinity();
  std::vector<double> mu(mu_inout, mu_inout + S), lo(S, -inf), hi(S, inf), N(S), dN(S);
  std::vector<double> best_mu(mu), best_f(S, inf);
  std::vector<char> done(S, 0);
  int it = 0;
  for (; it < max_iter;) {
    gf_status st = eval(mu.data(), N.data(), dN.data());
    ++it;
    if (st) return st;
    bool all = true;
    for (int s = 0; s < S; ++s) {
      if (done[s]) continue;
      const double f = N[s] - n_target[s];
      if (std::fabs(f) < best_f[s]) { best_f[s] = std::fabs(f); best_mu[s] = mu[s]; }
      if (std::fabs(f) <= tol) { done[s] = 1; continue; }
      all = false;
      if (f < 0) lo[s] = std::max(lo[s], mu[s]);
      else hi[s] = std::min(hi[s], mu[s]);
      double step = (dN[s] > 1e-300) ? -f / dN[s] : (f < 0 ? 1.0 : -1.0);
      const double cap = 4.0;  // eV: no wild jumps while the bracket is one-sided
      if (!(std::isfinite(lo[s]) && std::isfinite(hi[s]))) step = std::max(-cap, std::min(cap, step));
      double mn = mu[s] + step;
      if (std::isfinite(lo[s]) && std::isfinite(hi[s])) {
        if (!(mn > lo[s] && mn < hi[s])) mn = 0.5 * (lo[s] + hi[s]);
        if (hi[s] - lo[s] <= 4e-16 * std::max(1.0, std::fabs(mu[s]))) { done[s] = 2; continue; }
      }
      mu[s] = mn;
    }
    if (all) break;
  }
  bool conv = true;
  for (int s = 0; s < S; ++s) {
    if (done[s] != 1) conv = false;
    mu_inout[s] = done[s] == 1 ? mu[s] : best_mu[s];
  }
  if (iters_out) *iters_out = it;
  if (!conv) return fail(c, GF_ENOTCONV, "mu search did not reach tol within max_iter");
  return GF_OK;
}

}  // namespace gf_host

