// Mixed-precision N(mu) pass for small windows (N_b <= 40): one warp per matrix,
// the matrix in the warp's registers, no block barrier in the elimination.
//
// Per (k, i w_n) point, as the FP32 register kernel computes it (Eq. dmftloop1):
// A = (i w_n + mu) I - H_k - P_k^+ (Sigma(i w_n) P_k) in FP32 (the diagonal formed in
// FP64 and rounded once), X = A^{-1}, and Re Tr X, Re Tr X^2 summed over the item's
// frequencies in FP64 (the N(mu) and dN/dmu partial sums).
//
// The elimination (one warp per matrix, rows rotated one column per pivot, rows 32 to 39
// of 33- to 40-band windows split over four lanes, lazy row scales) is warp_invert of
// gf_warp_gj.cuh.  Windows of 41 to 96 bands run k_point_wm below: two or three warps
// per matrix, one row per lane.
#include <math.h>
#include <stdint.h>

#include "gf_complex.cuh"
#include "gf_internal.cuh"
#include "gf_warp_gj.cuh"

namespace gf {

namespace {

using namespace cx;
using wgj::pack_key_w;
using wgj::zero2;

}  // namespace

// Shared memory of k_point_w32 (bytes): per CTA P and H_ii of the item's k-point; per
// warp Sigma, T = Sigma P (then the inverse for the traces), the diagonal, the pivot
// row buffer and the pivot tables.
struct LayoutW {
  size_t oP, oHii, warp0, wstride, wS, wX, wD, wBuf, wPiv, bytes;
};

__host__ __device__ inline LayoutW make_layout_w(int nbmax, int mmax, int nmax, int nwarps) {
  auto al = [](size_t x) { return (x + 15) & ~(size_t)15; };
  LayoutW L;
  size_t o = 0;
  L.oP = o; o = al(o + 8 * (size_t)mmax * nbmax);
  L.oHii = o; o = al(o + 16 * (size_t)nbmax);
  L.warp0 = o;
  size_t g = 0;
  const size_t ld = (size_t)(nbmax | 1);
  size_t x = (size_t)mmax * nbmax;
  if (x < (size_t)nbmax * ld) x = (size_t)nbmax * ld;
  L.wS = g; g = al(g + 8 * (size_t)mmax * mmax);
  L.wX = g; g = al(g + 8 * x);
  L.wD = g; g = al(g + 8 * (size_t)nbmax);
  L.wBuf = g; g = al(g + 8 * (size_t)nmax);
  L.wPiv = g; g = al(g + 3 * sizeof(int) * (size_t)nmax);
  L.wstride = g;
  L.bytes = L.warp0 + (size_t)nwarps * g;
  return L;
}

// Shared memory of k_point_wm (bytes): P and H_ii of the item's k-point, Sigma, T =
// Sigma P (then the inverse for the traces), the diagonal, the double-buffered pivot
// row stage of every warp and the pivot tables.
struct LayoutM {
  size_t oP, oHii, oS, oX, oD, oStage, oPiv, bytes;
};

__host__ __device__ inline LayoutM make_layout_m(int nbmax, int mmax, int nmax) {
  auto al = [](size_t x) { return (x + 15) & ~(size_t)15; };
  LayoutM L;
  const size_t ld = (size_t)(nbmax | 1);
  size_t x = (size_t)mmax * nbmax;
  if (x < (size_t)nbmax * ld) x = (size_t)nbmax * ld;
  size_t o = 0;
  L.oP = o; o = al(o + 8 * (size_t)mmax * nbmax);
  L.oHii = o; o = al(o + 16 * (size_t)nbmax);
  L.oS = o; o = al(o + 8 * (size_t)mmax * mmax);
  L.oX = o; o = al(o + 8 * x);
  L.oD = o; o = al(o + 8 * (size_t)nbmax);
  L.oStage = o; o = al(o + 8 * 2 * (size_t)(nmax / 32) * nmax);
  L.oPiv = o; o = al(o + 3 * sizeof(int) * (size_t)nmax);
  L.bytes = o;
  return L;
}

namespace {

// 2-warp CTAs resident per SM that the register budget must allow (168 registers a
// thread); shared memory allows six for a 40-band window with 14 orbitals.
constexpr int kW32MinBlocks = 6;

template <int NMAX, int W, bool SPLIT>
__global__ void __launch_bounds__(32 * W, kW32MinBlocks) k_point_w32(const PointParams p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_item;
  __shared__ double s_part[W][2];
  const LayoutW L = make_layout_w(p.nbmax, p.mmax, NMAX, W);
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  float2* sP = reinterpret_cast<float2*>(smraw + L.oP);
  double2* sHii = reinterpret_cast<double2*>(smraw + L.oHii);
  unsigned char* wb = smraw + L.warp0 + (size_t)wp * L.wstride;
  float2* sS = reinterpret_cast<float2*>(wb + L.wS);
  float2* sX = reinterpret_cast<float2*>(wb + L.wX);
  float2* sD = reinterpret_cast<float2*>(wb + L.wD);
  int* sPiv = reinterpret_cast<int*>(wb + L.wPiv);
  const wgj::WarpBufs bufs{sX, reinterpret_cast<float2*>(wb + L.wBuf), sPiv, sPiv + NMAX, sPiv + 2 * NMAX};
  const int* sIdx = bufs.sIdx;
  const int* sRow = bufs.sRow;

  for (;;) {
    if (tid == 0) s_item = atomicAdd(p.queue, 1);
    __syncthreads();
    const int itx = s_item;
    if (itx >= p.n_items) break;
    const Item it = p.items[itx];
    const int kk = item_k(it, p.kperm, 0);  // N(mu) items hold one k-point
    const KInfo ki = p.kinfo[kk];
    const SInfo si = p.sinfo[ki.sys];
    const int N = ki.nb, M = si.m;
    const float2* Hk = p.Hs + ki.offH;
    const double2* Hk64 = p.H + ki.offH;
    const double mu = p.mu[ki.sys];
    const double pib = M_PI / si.beta;
    for (int e = tid; e < M * N; e += 32 * W) sP[e] = p.Ps[ki.offP + e];
    for (int x = tid; x < N; x += 32 * W) sHii[x] = Hk64[x * N + x];
    __syncthreads();
    double acc_tr = 0.0, acc_g2 = 0.0;

    for (int n = it.n0 + wp; n < it.n1; n += W) {
      const double wn = (2.0 * n + 1.0) * pib;
      wgj::warp_point_inputs(p.Ss + si.offSig + (int64_t)n * M * M, sHii, sP, mu, wn, N, M, lane, sS, sD, sX);
      wgj::warp_invert<NMAX, SPLIT>(Hk, sD, sP, bufs, N, M, lane, p.status);
      for (int x = lane; x < N; x += 32) acc_tr += (double)sX[sRow[x] + sIdx[x]].x;
      float g2 = 0.f;
      for (int e = lane; e < N * N; e += 32) {
        const int i = e / N, c = e - i * N;
        const float2 g1 = sX[sRow[i] + sIdx[c]], g3 = sX[sRow[c] + sIdx[i]];
        g2 = __fmaf_rn(g1.x, g3.x, __fmaf_rn(-g1.y, g3.y, g2));
      }
      acc_g2 += (double)g2;
      __syncwarp();  // sX and sS are rewritten by the next frequency
    }
    // deterministic: xor tree in each warp, then the warps in order
    for (int off = 16; off; off >>= 1) {
      acc_tr += __shfl_xor_sync(0xffffffffu, acc_tr, off);
      acc_g2 += __shfl_xor_sync(0xffffffffu, acc_g2, off);
    }
    if (lane == 0) {
      s_part[wp][0] = acc_tr;
      s_part[wp][1] = acc_g2;
    }
    __syncthreads();
    if (tid == 0) {
      double t = 0.0, u = 0.0;
      for (int w = 0; w < W; ++w) {
        t += s_part[w][0];
        u += s_part[w][1];
      }
      double* o = p.occ_part + ((int64_t)kk * p.n_chunks + it.chunk) * 2;
      o[0] = t;
      o[1] = u;
    }
    __syncthreads();
  }
}

// Windows of 41 to 96 bands: WPM warps per matrix, one row per lane (row 32 w + lane),
// the same rotated exchange-form elimination with lazy row scales.  Per pivot every
// warp's best unused row stages its values and key (double-buffered), one CTA barrier,
// then every thread takes the group's winner from the stage.
template <int NMAX, int WPM>
__global__ void __launch_bounds__(32 * WPM) k_point_wm(const PointParams p) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_item;
  __shared__ unsigned s_key[2][4];
  __shared__ double s_red[WPM];
  const LayoutM L = make_layout_m(p.nbmax, p.mmax, NMAX);
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int r = tid;  // this thread's row
  float2* sP = reinterpret_cast<float2*>(smraw + L.oP);
  double2* sHii = reinterpret_cast<double2*>(smraw + L.oHii);
  float2* sS = reinterpret_cast<float2*>(smraw + L.oS);
  float2* sX = reinterpret_cast<float2*>(smraw + L.oX);
  float2* sD = reinterpret_cast<float2*>(smraw + L.oD);
  float2* sStage = reinterpret_cast<float2*>(smraw + L.oStage);  // [2][WPM][NMAX]
  int* sPiv = reinterpret_cast<int*>(smraw + L.oPiv);
  int* sIdx = sPiv + NMAX;
  int* sRow = sIdx + NMAX;

  for (;;) {
    if (tid == 0) s_item = atomicAdd(p.queue, 1);
    __syncthreads();
    const int itx = s_item;
    if (itx >= p.n_items) break;
    const Item it = p.items[itx];
    const int kk = item_k(it, p.kperm, 0);  // N(mu) items hold one k-point
    const KInfo ki = p.kinfo[kk];
    const SInfo si = p.sinfo[ki.sys];
    const int N = ki.nb, M = si.m, ld = N | 1;
    const float2* Hk = p.Hs + ki.offH;
    const double2* Hk64 = p.H + ki.offH;
    const double mu = p.mu[ki.sys];
    const double pib = M_PI / si.beta;
    for (int e = tid; e < M * N; e += 32 * WPM) sP[e] = p.Ps[ki.offP + e];
    for (int x = tid; x < N; x += 32 * WPM) sHii[x] = Hk64[x * N + x];
    double acc_tr = 0.0, acc_g2 = 0.0;

    for (int n = it.n0; n < it.n1; ++n) {
      const double wn = (2.0 * n + 1.0) * pib;
      __syncthreads();  // sP, sHii loaded; the previous frequency is done with sX, sS
      for (int e = tid; e < M * M; e += 32 * WPM) sS[e] = p.Ss[si.offSig + (int64_t)n * M * M + e];
      for (int x = tid; x < N; x += 32 * WPM)
        sD[x] = make_float2(__double2float_rn(mu - sHii[x].x), __double2float_rn(wn - sHii[x].y));
      __syncthreads();
      for (int e = tid; e < M * N; e += 32 * WPM) {  // T = Sigma P (M x N)
        const int a = e / N, j = e - a * N;
        float2 acc = zero2();
        for (int b = 0; b < M; ++b) fmac(acc, sS[a * M + b], sP[b * N + j]);
        sX[e] = acc;
      }
      __syncthreads();
      float2 a[NMAX];
#pragma unroll
      for (int c = 0; c < NMAX; ++c) {
        float2 v = zero2();
        if (r < N && c < N) {
          const float2 h = Hk[r * N + c];
          v = (r == c) ? sD[r] : make_float2(-h.x, -h.y);
        }
        a[c] = v;
      }
      if (r < N) {
        for (int x = 0; x < M; ++x) {
          const float2 pv = sP[x * N + r];
          const float2 mp = make_float2(-pv.x, pv.y);  // -conj(P[x][r])
#pragma unroll
          for (int c = 0; c < NMAX; ++c)
            if (c < N) fmac(a[c], mp, sX[x * N + c]);
        }
      }
      bool used = false;
      float2 sc = make_float2(1.f, 0.f);
      int par = 0;
#pragma unroll 1
      for (int j = 0; j < N; ++j) {
        const unsigned key = (r < N && !used) ? pack_key_w(a[0], r) : 0u;
        const unsigned wk = __reduce_max_sync(0xffffffffu, key);
        float2* stg = sStage + (par * WPM + wp) * NMAX;
        if (wk != 0u && r == 127 - (int)(wk & 127u)) {
#pragma unroll
          for (int c = 0; c < NMAX; c += 2)
            *reinterpret_cast<float4*>(stg + c) = make_float4(a[c].x, a[c].y, a[c + 1].x, a[c + 1].y);
          s_key[par][wp] = wk;
        } else if (wk == 0u && lane == 0) {
          s_key[par][wp] = 0u;
        }
        __syncthreads();
        unsigned best = s_key[par][0];
        int qw = 0;
#pragma unroll
        for (int x = 1; x < WPM; ++x) {
          const unsigned kx = s_key[par][x];
          if (kx > best) {
            best = kx;
            qw = x;
          }
        }
        const int prow = min(127 - (int)(best & 127u), N - 1);
        if (tid == 0) {
          if ((best >> 7) == 0u || (best & ~127u) >= 0x7f800000u) atomicOr(p.status, kFlagSingular);
          sPiv[j] = prow;
        }
        const float2* u = sStage + (par * WPM + qw) * NMAX;
        const float2 rc = frcp(u[0]);
        const bool isp = (r == prow);
        const float2 lq = isp ? zero2() : fmul(a[0], rc);
#pragma unroll
        for (int c = 1; c < NMAX; ++c) fsub_prod(a[c], lq, u[c]);
        const float2 col = isp ? make_float2(1.f, 0.f) : make_float2(-lq.x, -lq.y);
#pragma unroll
        for (int c = 0; c + 1 < NMAX; ++c) a[c] = a[c + 1];
        a[NMAX - 1] = col;
        if (isp) {
          used = true;
          sc = rc;
        }
        par ^= 1;
      }
      __syncthreads();  // every thread is done with the stage and sX before the dump
      if (r < N)
#pragma unroll
        for (int x = 0; x < NMAX; ++x) {
          int c = x + N;
          if (c >= NMAX) c -= NMAX;
          if (c < N) sX[r * ld + c] = fmul(sc, a[x]);
        }
      for (int j = tid; j < N; j += 32 * WPM) sIdx[sPiv[j]] = j;
      __syncthreads();
      for (int x = tid; x < N; x += 32 * WPM) sRow[x] = sPiv[x] * ld;
      __syncthreads();
      for (int x = tid; x < N; x += 32 * WPM) acc_tr += (double)sX[sRow[x] + sIdx[x]].x;
      float g2 = 0.f;
      for (int e = tid; e < N * N; e += 32 * WPM) {
        const int i = e / N, c = e - i * N;
        const float2 g1 = sX[sRow[i] + sIdx[c]], g3 = sX[sRow[c] + sIdx[i]];
        g2 = __fmaf_rn(g1.x, g3.x, __fmaf_rn(-g1.y, g3.y, g2));
      }
      acc_g2 += (double)g2;
    }
    // deterministic: xor tree in each warp, then the warps in order
    for (int off = 16; off; off >>= 1) {
      acc_tr += __shfl_xor_sync(0xffffffffu, acc_tr, off);
      acc_g2 += __shfl_xor_sync(0xffffffffu, acc_g2, off);
    }
    __syncthreads();
    if (lane == 0) s_red[wp] = acc_tr;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < WPM; ++w) t += s_red[w];
    __syncthreads();
    if (lane == 0) s_red[wp] = acc_g2;
    __syncthreads();
    if (tid == 0) {
      double u2 = 0.0;
      for (int w = 0; w < WPM; ++w) u2 += s_red[w];
      double* o = p.occ_part + ((int64_t)kk * p.n_chunks + it.chunk) * 2;
      o[0] = t;
      o[1] = u2;
    }
    __syncthreads();
  }
}

template <int NMAX, int WPM>
cudaError_t launch_m(const PointParams& p, int grid, size_t smem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_point_wm<NMAX, WPM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_point_wm<NMAX, WPM><<<grid, 32 * WPM, smem, s>>>(p);
  return cudaGetLastError();
}

template <int NMAX, int WPM>
int bps_m(size_t smem) {
  int nb = 0;
  if (cudaFuncSetAttribute(k_point_wm<NMAX, WPM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_point_wm<NMAX, WPM>, 32 * WPM, smem) != cudaSuccess)
    return 0;
  return nb;
}

constexpr int kW32Warps = 2;  // warps (matrices in flight) per CTA

// Dynamic shared memory of the launch, and the largest carveout: six 2-warp CTAs of a
// 40-band window (36 KB each) fill an SM only with the whole 228 KB as shared memory.
template <int NMAX, bool SPLIT>
cudaError_t set_attrs_w(size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(k_point_w32<NMAX, kW32Warps, SPLIT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_point_w32<NMAX, kW32Warps, SPLIT>,
                              cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
}

template <int NMAX, bool SPLIT>
cudaError_t launch_w(const PointParams& p, int grid, size_t smem, cudaStream_t s) {
  const cudaError_t e = set_attrs_w<NMAX, SPLIT>(smem);
  if (e != cudaSuccess) return e;
  k_point_w32<NMAX, kW32Warps, SPLIT><<<grid, 32 * kW32Warps, smem, s>>>(p);
  return cudaGetLastError();
}

template <int NMAX, bool SPLIT>
int bps_w(size_t smem) {
  int nb = 0;
  if (set_attrs_w<NMAX, SPLIT>(smem) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_point_w32<NMAX, kW32Warps, SPLIT>,
                                                    32 * kW32Warps, smem) != cudaSuccess)
    return 0;
  return nb;
}

}  // namespace

// Largest window of the instantiation that serves nbmax, or 0.
int w32_nmax(int nbmax) { return nbmax <= 16 ? 16 : (nbmax <= 32 ? 32 : (nbmax <= 40 ? 40 : 0)); }

// Multi-warp form: windows of 41 to 96 bands, 2 or 3 warps per matrix.
int wm_nmax(int nbmax) { return nbmax <= 40 ? 0 : (nbmax <= 64 ? 64 : (nbmax <= 96 ? 96 : 0)); }

int wm_threads(int nbmax) { return wm_nmax(nbmax); }

size_t point_wm_smem(int nbmax, int mmax) { return make_layout_m(nbmax, mmax, wm_nmax(nbmax)).bytes; }

int point_wm_blocks_per_sm(int nbmax, size_t smem) {
  switch (wm_nmax(nbmax)) {
    case 64: return bps_m<64, 2>(smem);
    case 96: return bps_m<96, 3>(smem);
    default: return 0;
  }
}

cudaError_t launch_point_wm(int nbmax, const PointParams& p, int grid, size_t smem, cudaStream_t s) {
  switch (wm_nmax(nbmax)) {
    case 64: return launch_m<64, 2>(p, grid, smem, s);
    case 96: return launch_m<96, 3>(p, grid, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

int w32_threads() { return 32 * kW32Warps; }

size_t point_w32_smem(int nbmax, int mmax) {
  return make_layout_w(nbmax, mmax, w32_nmax(nbmax), kW32Warps).bytes;
}

int point_w32_blocks_per_sm(int nbmax, size_t smem) {
  switch (w32_nmax(nbmax)) {
    case 16: return bps_w<16, false>(smem);
    case 32: return bps_w<32, false>(smem);
    case 40: return bps_w<40, true>(smem);
    default: return 0;
  }
}

cudaError_t launch_point_w32(int nbmax, const PointParams& p, int grid, size_t smem, cudaStream_t s) {
  switch (w32_nmax(nbmax)) {
    case 16: return launch_w<16, false>(p, grid, smem, s);
    case 32: return launch_w<32, false>(p, grid, smem, s);
    case 40: return launch_w<40, true>(p, grid, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gf
