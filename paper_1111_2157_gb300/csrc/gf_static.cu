// gf_occupation_static: N(mu) and dN/dmu for one uniform system without any
// device allocation.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool or allocator hooks, plugins that must not grow the
// device footprint after start-up, and hosts that forbid allocation on their
// hot path.  For them this entry point keeps all of its scratch (work queue,
// status word, k/system/item tables, per-(k, chunk) partial sums, per-k traces
// and the two results) in the file-scope device array g_scratch below, of a
// fixed size of kStaticScratchBytes.  Every GPU that loads the library holds
// that array until the process exits.  The caller passes the inputs and gets
// the outputs; the same point kernel as gf_occupation does the work.
#include <algorithm>
#include <cmath>

#include "gf.h"
#include "gf_internal.cuh"

namespace {

constexpr size_t kStaticScratchBytes = (size_t)4 << 20;  // 4 MiB per device

static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct StaticLayout {
  size_t counters, kinfo, sinfo, items, occ, trHE, kN, kdN, mu, out, bytes;
};

StaticLayout static_layout(int n_k, int n_items) {
  StaticLayout L;
  size_t o = 0;
  L.counters = o; o = align256(o + 2 * sizeof(int));  // [0] work queue, [1] status
  L.kinfo = o; o = align256(o + sizeof(gf::KInfo) * (size_t)n_k);
  L.sinfo = o; o = align256(o + sizeof(gf::SInfo));
  L.items = o; o = align256(o + sizeof(gf::Item) * (size_t)n_items);
  L.occ = o; o = align256(o + 2 * sizeof(double) * (size_t)n_items);
  L.trHE = o; o = align256(o + sizeof(double) * (size_t)n_k);
  L.kN = o; o = align256(o + sizeof(double) * (size_t)n_k);
  L.kdN = o; o = align256(o + sizeof(double) * (size_t)n_k);
  L.mu = o; o = align256(o + sizeof(double));
  L.out = o; o = align256(o + 2 * sizeof(double));
  L.bytes = o;
  return L;
}

// Tables of one uniform system and trHE_k = Re Tr H_k + Re Tr(Sigma_inf P_k P_k^+) (the same
// trhe_partial as the context path).  One CTA per k.
__global__ void __launch_bounds__(256) k_static_setup(
    const double2* __restrict__ H, const double2* __restrict__ P, const double2* __restrict__ Sinf,
    int n_k, int nb, int m, int n_chunks, int chunk_w, int n_iw, double beta, double tailc, double mu,
    gf::KInfo* __restrict__ kinfo, gf::SInfo* __restrict__ sinfo, gf::Item* __restrict__ items,
    double* __restrict__ trHE, double* __restrict__ mu_out) {
  __shared__ double red[8];
  const int k = blockIdx.x;
  if (threadIdx.x == 0) {
    gf::KInfo ki;
    ki.nb = nb;
    ki.sys = 0;
    ki.offH = (int64_t)k * nb * nb;
    ki.offP = (int64_t)k * m * nb;
    ki.w = 1.0 / n_k;
    kinfo[k] = ki;
    if (k == 0) {
      gf::SInfo si;
      si.m = m;
      si.k0 = 0;
      si.k1 = n_k;
      si.pad = 0;
      si.beta = beta;
      si.tailc = tailc;
      si.offSig = 0;
      si.offSinf = 0;
      sinfo[0] = si;
      *mu_out = mu;
    }
  }
  for (int ch = threadIdx.x; ch < n_chunks; ch += blockDim.x) {
    gf::Item it;
    it.k = k;
    it.n0 = ch * chunk_w;
    it.n1 = min(n_iw, (ch + 1) * chunk_w);
    it.chunk = ch;
    it.nk = 1;
    it.g = k;
    items[(int64_t)k * n_chunks + ch] = it;
  }
  double v = gf::trhe_partial(H + (int64_t)k * nb * nb, P + (int64_t)k * m * nb, Sinf, nb, m,
                              threadIdx.x, blockDim.x);
  for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    trHE[k] = t;
  }
}

// Device address of g_scratch on the current device.  Looked up on every call (about a
// microsecond): a cached address would go stale after cudaDeviceReset or when another
// context becomes current on the device, and the module is then loaded afresh.
gf_status scratch_for_current_device(unsigned char** out) {
  void* ptr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
  if (e != cudaSuccess || !ptr) {
    gf::set_global_error(e != cudaSuccess ? cudaGetErrorString(e)
                                          : "gf_occupation_static: no device address for the scratch");
    return GF_ECUDA;
  }
  *out = static_cast<unsigned char*>(ptr);
  return GF_OK;
}

#define GF_SCU(call)                                                                  \
  do {                                                                                \
    const cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess) {                                                          \
      gf::set_global_error(cudaGetErrorString(e_));                                   \
      return GF_ECUDA;                                                                \
    }                                                                                 \
  } while (0)

}  // namespace

extern "C" gf_status gf_occupation_static(const void* h_dev, const void* p_dev, const void* sigma_dev,
                                          const void* sigma_inf_dev, int32_t n_k, int32_t nb,
                                          int32_t m, int32_t n_iw, double beta, double mu,
                                          int32_t tail_order, void* stream, double* n_out,
                                          double* dn_dmu_out) try {
  gf::set_global_error("");
  if (!h_dev || !p_dev || !sigma_dev || !sigma_inf_dev || !n_out) {
    gf::set_global_error("gf_occupation_static: NULL input or n_out");
    return GF_EINVAL;
  }
  if (n_k < 1 || nb < 1 || m < 1 || n_iw < 1 || !(beta > 0.0) || !std::isfinite(beta) ||
      !std::isfinite(mu) || (tail_order != 1 && tail_order != 2)) {
    gf::set_global_error("gf_occupation_static: invalid sizes, beta, mu or tail_order");
    return GF_EINVAL;
  }
  unsigned char* base = nullptr;
  gf_status st = scratch_for_current_device(&base);
  if (st) return st;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0, optin = 0;
  GF_SCU(cudaGetDevice(&dev));
  GF_SCU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  GF_SCU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const size_t smem = gf::point_fp64_smem(nb, m, gf::kOcc, 1);
  if (smem > (size_t)optin - 1024) {
    gf::set_global_error("gf_occupation_static: N_b or m too large for shared memory");
    return GF_EINVAL;
  }
  int bps = gf::point_fp64_blocks_per_sm(smem);
  if (bps < 1) bps = 1;
  const int grid_max = sms * bps;
  // about 40 items per resident CTA, at least 4 frequencies per item
  const double want = (double)n_k * n_iw / (40.0 * grid_max);
  const int chunk_w = (int)std::min<double>(n_iw, std::max(4.0, std::ceil(want)));
  const int n_chunks = (n_iw + chunk_w - 1) / chunk_w;
  const int64_t n_items64 = (int64_t)n_k * n_chunks;
  const StaticLayout L = static_layout(n_k, (int)std::min<int64_t>(n_items64, 1 << 30));
  if (n_items64 > (1 << 30) || L.bytes > kStaticScratchBytes) {
    gf::set_global_error("gf_occupation_static: problem exceeds the 4 MiB static scratch "
                         "(n_k * ceil(n_iw / chunk) items of 32 B plus 56 B per k)");
    return GF_EINVAL;
  }
  const int n_items = (int)n_items64;
  int* counters = reinterpret_cast<int*>(base + L.counters);
  gf::KInfo* kinfo = reinterpret_cast<gf::KInfo*>(base + L.kinfo);
  gf::SInfo* sinfo = reinterpret_cast<gf::SInfo*>(base + L.sinfo);
  gf::Item* items = reinterpret_cast<gf::Item*>(base + L.items);
  double* occ = reinterpret_cast<double*>(base + L.occ);
  double* trHE = reinterpret_cast<double*>(base + L.trHE);
  double* kN = reinterpret_cast<double*>(base + L.kN);
  double* kdN = reinterpret_cast<double*>(base + L.kdN);
  double* mu_d = reinterpret_cast<double*>(base + L.mu);
  double* out = reinterpret_cast<double*>(base + L.out);

  // The work queue and the status word must start at zero; the rest is overwritten.
  GF_SCU(cudaMemsetAsync(counters, 0, 2 * sizeof(int), s));
  const double tailc = gf::tail_coefficient(beta, n_iw, tail_order);
  k_static_setup<<<n_k, 256, 0, s>>>(static_cast<const double2*>(h_dev),
                                     static_cast<const double2*>(p_dev),
                                     static_cast<const double2*>(sigma_inf_dev), n_k, nb, m, n_chunks,
                                     chunk_w, n_iw, beta, tailc, mu, kinfo, sinfo, items, trHE, mu_d);
  GF_SCU(cudaGetLastError());
  gf::PointParams p{};
  p.H = static_cast<const double2*>(h_dev);
  p.P = static_cast<const double2*>(p_dev);
  p.Sig = static_cast<const double2*>(sigma_dev);
  p.kinfo = kinfo;
  p.sinfo = sinfo;
  p.items = items;
  p.n_items = n_items;
  p.n_chunks = n_chunks;
  p.queue = counters;
  p.mu = mu_d;
  p.mode = gf::kOcc;
  p.nbmax = nb;
  p.mmax = m;
  p.a_in_smem = 1;
  p.occ_part = occ;
  p.n_iw = n_iw;
  p.status = counters + 1;
  GF_SCU(gf::launch_point_fp64(p, std::min(grid_max, n_items), smem, s));
  GF_SCU(gf::launch_occ_finalize(kinfo, sinfo, trHE, mu_d, occ, n_chunks, n_k, kN, kdN, s));
  GF_SCU(gf::launch_sys_reduce(kinfo, sinfo, 1, kN, kdN, out, s));
  double res[2] = {0.0, 0.0};
  int status = 0;
  GF_SCU(cudaMemcpyAsync(res, out, sizeof(res), cudaMemcpyDeviceToHost, s));
  GF_SCU(cudaMemcpyAsync(&status, counters + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  GF_SCU(cudaStreamSynchronize(s));
  if (status & gf::kFlagSingular) {
    gf::set_global_error("gf_occupation_static: zero or non-finite pivot");
    return GF_ESINGULAR;
  }
  *n_out = res[0];
  if (dn_dmu_out) *dn_dmu_out = res[1];
  return GF_OK;
} catch (...) {
  return gf::caught_global();
}
