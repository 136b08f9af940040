// Mixed-precision N(mu) pass on the tcgen05 tensor cores (sm_103a): blocked
// Gauss-Jordan inverse with the matrix resident in tensor memory.
//
// Per (k, i w_n) point, as the FP32 register kernel computes it (Eq. dmftloop1):
//   A = (i w_n + mu) I - H_k - P_k^+ (Sigma(i w_n) P_k) in FP32 (the diagonal
//   formed in FP64 and rounded once), X = A^{-1}, and Re Tr X, Re Tr X^2 summed
//   over the item's frequencies in FP64 (the N(mu) and dN/dmu partial sums).
//
// Elimination.  Gauss-Jordan in exchange (sweep) form with partial pivoting:
// pivot step j sweeps (p_j, j), p_j the unused row of largest |M[i][j]|; after
// all steps X[i][c] = M[p_i][q_c], q the inverse permutation of p.  Sweeping a
// block of b pivots (rows P, columns Q) at once is
//   M'[:, Q] = the b sequential sweeps applied to the panel columns only,
//   M'[:, J] = M[:, J] + L M[P, J]          (J = the other columns)
// with L = M'[:, Q] minus 1 at (p_t, q_t): column t of L pairs with old row
// p_t.  So each block is a panel factorisation of an N x b column block (CUDA
// cores, registers, one barrier per pivot) and one rank-b update of the whole
// matrix, which is a GEMM: D(128 x 2N) += A_op(128 x 2b) B_op(2N x 2b)^T with
// real operands [Re L | Im L] and [[Re R, -Im R], [Im R, Re R]] (R = old pivot
// rows), D = [Re M | Im M] in tensor memory.  The GEMM runs as tcgen05.mma
// kind::tf32 with FP32 accumulation; each operand is split x = hi + lo into two
// TF32 values rounded to nearest (11 significant bits each, |x - hi - lo| <=
// 2^-22 |x|), and hi*hi + hi*lo + lo*hi gives products to about 2^-22 relative,
// near the FP32 elimination's 2^-24.
// Windows are padded to a multiple of 8 with an identity block, which stays
// decoupled from the real block and pivots on itself.
//
// CTA layout: NG groups of 4 warps; warp q of a group owns tensor-memory lanes
// 32q..32q+31, i.e. rows 32q + lane of its group's matrix and of its A operand
// (hi and lo TF32 parts of [Re L | Im L], next to the matrix in tensor memory).  The groups share the
// work item's k-point and take its frequencies in turn.  One thread per group
// issues the group's MMAs and commits them to the group's mbarrier; every wait
// on it is bounded (on timeout the kernel flags kFlagTimeout and stops taking
// work).  Operands in shared memory use the canonical K-major layout without
// swizzling: 8-row x 16-byte core matrices, 128 B apart along K and 1 KiB apart
// along the rows (K = 32 values per row).
#include <math.h>
#include <stdint.h>

#include "gf_complex.cuh"
#include "gf_internal.cuh"

namespace gf {

namespace {

using namespace cx;

constexpr int kTcB = 16;                          // pivots per block
constexpr int kTcK = 2 * kTcB;                    // GEMM depth per block (real and imaginary parts)
constexpr uint32_t kKChunk = 128;                 // bytes between K-adjacent core matrices
constexpr uint32_t kRowGroup = 128 * (kTcK / 4);  // bytes between 8-row groups (1 KiB)
constexpr long kWaitLimit = 1L << 20;             // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (r, k) of a K-major operand (K = kTcK).
__device__ __forceinline__ uint32_t op_off(int r, int k) {
  return (uint32_t)((r & 7) * 16 + (k & 3) * 4) + (uint32_t)(k >> 2) * kKChunk + (uint32_t)(r >> 3) * kRowGroup;
}

// Shared-memory matrix descriptor: start, leading (K) and stride (row-group)
// byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((kKChunk >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((kRowGroup >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, M = 128, N = n.
__device__ __forceinline__ uint32_t mma_idesc(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// D += A B^T with A in tensor memory (row i = lane i, K consecutive columns).
__device__ __forceinline__ void mma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, 1, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}

// Bounded wait for the completion of phase `parity` of an mbarrier.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_addr(bar);
  for (long it = 0; it < kWaitLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void group_bar(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }

__device__ __forceinline__ void tmem_ld8(uint32_t ta, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(ta));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_st8(uint32_t ta, const float (&v)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(ta),
               "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
               "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
               "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
               : "memory");
}

// x rounded to the nearest TF32 value (11 significant bits)
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// x = hi + lo with hi and lo TF32 values: |x - hi - lo| <= 2^-22 |x|
__device__ __forceinline__ void put_split(unsigned char* hi, unsigned char* lo, uint32_t off, float x) {
  const float h = tf32_rna(x);
  *reinterpret_cast<float*>(hi + off) = h;
  *reinterpret_cast<float*>(lo + off) = tf32_rna(x - h);
}

__device__ __forceinline__ void tmem_ld16(uint32_t ta, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(ta));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Pivot key with the row index (< 128) in its low 7 bits: largest |.| wins, ties
// go to the lowest row.
__device__ __forceinline__ unsigned pack_key_tc(float2 v, int i) {
  return (pivot_key_s(v) & ~127u) | (unsigned)(127 - i);
}

__device__ __forceinline__ double block_sum_tc(double v, double* red) {
  // Deterministic: fixed xor tree in each warp, then warp 0 over the warps.
  for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (warp == 0) {
    r = lane < nw ? red[lane] : 0.0;
    for (int off = 16; off; off >>= 1) r += __shfl_xor_sync(0xffffffffu, r, off);
  }
  return r;
}

}  // namespace

// Shared-memory layout of k_point_tc (bytes): per CTA P and H_ii of the item's
// k-point; per group the operand region (B_op hi/lo, and after it Sigma and
// T = Sigma P, which the embedding uses before the first block; after the last
// block the region holds the inverse for the traces), the diagonal, pivot tables
// and the staging buffers.  A_op lives in tensor memory.
struct LayoutTc {
  size_t oP, oHii, group0, gstride;
  size_t gOps, gBhi, gBlo, gS, gT, gD, gPiv, gStage, gKey, gWst, bytes;
};

__host__ __device__ inline int tc_np(int n) { return (n + 7) & ~7; }

__host__ __device__ inline size_t tc_align(size_t x, size_t a) { return (x + a - 1) & ~(a - 1); }

__host__ __device__ inline LayoutTc make_layout_tc(int nbmax, int mmax, int ng) {
  LayoutTc L;
  const int np = tc_np(nbmax);
  const size_t ld = (size_t)(nbmax | 1);
  size_t o = 0;
  L.oP = o; o = tc_align(o + 8 * (size_t)mmax * nbmax, 16);
  L.oHii = o; o = tc_align(o + 16 * (size_t)nbmax, 1024);
  L.group0 = o;
  const size_t b_bytes = 2 * (size_t)np * kTcK * 4;
  L.gOps = 0;
  L.gBhi = 0;
  L.gBlo = b_bytes;
  size_t g = 2 * b_bytes;
  L.gS = g; g = tc_align(g + 8 * (size_t)mmax * mmax, 16);
  L.gT = g; g = tc_align(g + 8 * (size_t)mmax * np, 16);  // [m][Np], zero beyond N
  const size_t dump = 8 * (size_t)nbmax * ld;
  if (dump > g) g = dump;
  g = tc_align(g, 16);
  L.gD = g; g = tc_align(g + 8 * (size_t)np, 16);
  L.gPiv = g; g = tc_align(g + 3 * sizeof(int) * (size_t)np, 16);
  L.gStage = g; g = tc_align(g + 2 * 4 * (size_t)kTcK * 4, 16);  // [2 buffers][4 warps][2b floats]
  L.gKey = g; g = tc_align(g + 2 * 4 * sizeof(unsigned), 16);      // [2 buffers][4 warps]
  L.gWst = g; g = tc_align(g + 4 * (size_t)kTcB * 17 * 4, 16);     // [4 warps][16 slots x 16 floats, 16 slot ids]
  L.gstride = tc_align(g, 1024);
  L.bytes = L.group0 + (size_t)ng * L.gstride;
  return L;
}

// Tensor-memory columns of one group (Re and Im planes of the padded matrix, then
// A_op hi and lo, kTcK columns each), rounded to 32, and of the CTA's allocation
// (a power of two, >= 32).
__host__ __device__ inline int tc_group_cols(int nbmax) { return (2 * tc_np(nbmax) + 2 * kTcK + 31) & ~31; }
__host__ __device__ inline int tc_alloc_cols(int nbmax, int ng) {
  const int need = ng * tc_group_cols(nbmax);
  int c = 32;
  while (c < need) c <<= 1;
  return c;
}

namespace {

// Panel factorisation of one block: BW sequential sweeps of the Np x BW column
// block held in (vr, vi), one row per thread.  Per pivot: each warp's best unused
// row stages its panel entries and key; one group barrier; every thread picks the
// group's winner, reads its row and applies the sweep (the pivot row takes l = -1
// and starts from zero, every other row zeroes its pivot-column entry; then
// v -= l w with w = u r and w_t = r, r = 1/u_t).  Warps without live rows only
// publish a zero key.
template <int BW>
__device__ __forceinline__ void panel_sweep(float (&vr)[kTcB], float (&vi)[kTcB], unsigned& used, int& my_t,
                                            int i, int Np, int q, int lane, int g, int gt, int j0, int& buf,
                                            bool live, float* sStage, unsigned* sKey, int* sPiv, int* status) {
#pragma unroll
  for (int t = 0; t < BW; ++t) {
    const float2 vt = make_float2(vr[t], vi[t]);
    unsigned wk = 0u;
    if (live) {
      const unsigned key = (i < Np && !used) ? pack_key_tc(vt, i) : 0u;
      wk = __reduce_max_sync(0xffffffffu, key);
      if (wk != 0u && i == 127 - (int)(wk & 127u)) {
        float* stg = sStage + (buf * 4 + q) * kTcK;
#pragma unroll
        for (int j = 0; j < BW; j += 4) {
          *reinterpret_cast<float4*>(stg + j) = make_float4(vr[j], vr[j + 1], vr[j + 2], vr[j + 3]);
          *reinterpret_cast<float4*>(stg + kTcB + j) = make_float4(vi[j], vi[j + 1], vi[j + 2], vi[j + 3]);
        }
        sKey[buf * 4 + q] = wk;
      }
    }
    if (wk == 0u && lane == 0) sKey[buf * 4 + q] = 0u;
    group_bar(1 + g);
    const uint4 k4 = *reinterpret_cast<const uint4*>(sKey + buf * 4);
    unsigned best = k4.x;
    int qw = 0;
    if (k4.y > best) { best = k4.y; qw = 1; }
    if (k4.z > best) { best = k4.z; qw = 2; }
    if (k4.w > best) { best = k4.w; qw = 3; }
    const int prow = 127 - (int)(best & 127u);
    if (gt == 0) {
      if ((best >> 7) == 0u || (best & ~127u) >= 0x7f800000u) atomicOr(status, kFlagSingular);
      sPiv[j0 + t] = min(prow, Np - 1);
    }
    if (live) {
      const float* ps = sStage + (buf * 4 + qw) * kTcK;
      float2 u[BW];
#pragma unroll
      for (int j = 0; j < BW; j += 4) {
        const float4 a4 = *reinterpret_cast<const float4*>(ps + j);
        const float4 b4 = *reinterpret_cast<const float4*>(ps + kTcB + j);
        u[j] = make_float2(a4.x, b4.x);
        u[j + 1] = make_float2(a4.y, b4.y);
        u[j + 2] = make_float2(a4.z, b4.z);
        u[j + 3] = make_float2(a4.w, b4.w);
      }
      const float2 r = frcp(u[t]);
      float2 l = vt;
      if (i == prow) {
        l = make_float2(-1.f, 0.f);
#pragma unroll
        for (int j = 0; j < BW; ++j) vr[j] = vi[j] = 0.f;
        used = 1u;
        my_t = t;
      } else {
        vr[t] = vi[t] = 0.f;
      }
#pragma unroll
      for (int j = 0; j < BW; ++j) {
        const float2 w = (j == t) ? r : fmul(u[j], r);
        float2 v = make_float2(vr[j], vi[j]);
        fsub_prod(v, l, w);
        vr[j] = v.x;
        vi[j] = v.y;
      }
    }
    buf ^= 1;
  }
}

template <int NG>
__global__ void __launch_bounds__(NG * 128, 1) k_point_tc(const PointParams p) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ __align__(8) uint64_t s_bar[NG];
  __shared__ uint32_t s_tmem;
  __shared__ int s_item, s_abort;
  __shared__ int s_fail[NG];
  __shared__ double s_red[NG * 4];
  const LayoutTc L = make_layout_tc(p.nbmax, p.mmax, NG);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = warp >> 2, q = warp & 3, gt = tid & 127;  // group, lane quadrant, thread in group
  const int i = 32 * q + lane;                              // this thread's matrix row
  float2* sP = reinterpret_cast<float2*>(smraw + L.oP);
  double2* sHii = reinterpret_cast<double2*>(smraw + L.oHii);
  unsigned char* gb = smraw + L.group0 + (size_t)g * L.gstride;
  unsigned char* bHi = gb + L.gBhi;
  unsigned char* bLo = gb + L.gBlo;
  float2* sG = reinterpret_cast<float2*>(gb + L.gOps);
  float2* sS = reinterpret_cast<float2*>(gb + L.gS);
  float2* sT = reinterpret_cast<float2*>(gb + L.gT);
  float2* sD = reinterpret_cast<float2*>(gb + L.gD);
  int* sPiv = reinterpret_cast<int*>(gb + L.gPiv);
  const int np_max = tc_np(p.nbmax);
  int* sIdx = sPiv + np_max;
  int* sRow = sIdx + np_max;
  float* sStage = reinterpret_cast<float*>(gb + L.gStage);
  unsigned* sKey = reinterpret_cast<unsigned*>(gb + L.gKey);
  float* sWst = reinterpret_cast<float*>(gb + L.gWst) + q * kTcB * 17;
  int* sSlotT = reinterpret_cast<int*>(sWst + kTcB * 16);
  const int gcols = tc_group_cols(p.nbmax);
  const int acols = tc_alloc_cols(p.nbmax, NG);

  // Zero the operand region once (entries that meet zero factors must be finite).
  for (int e = gt; e < 4 * np_max * kTcK; e += 128) reinterpret_cast<float*>(bHi)[e] = 0.f;
  if (tid == 0) {
    s_abort = 0;
    for (int x = 0; x < NG; ++x) s_fail[x] = 0;
    for (int x = 0; x < NG; ++x)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&s_bar[x])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                 "r"(acols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  proxy_fence();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem + (uint32_t)(g * gcols);       // this group's column 0
  const uint32_t tlane = tmem + ((uint32_t)(32 * q) << 16);  // this warp's lanes
  const uint32_t acol = (uint32_t)(2 * np_max);              // A_op hi at acol, lo at acol + kTcK
  uint32_t phase = 0;
  bool ok = true;

  for (;;) {
    if (tid == 0) s_item = s_abort ? p.n_items : atomicAdd(p.queue, 1);
    __syncthreads();
    const int itx = s_item;
    if (itx >= p.n_items) break;
    const Item it = p.items[itx];
    const int kk = item_k(it, p.kperm, 0);
    const KInfo ki = p.kinfo[kk];
    const SInfo si = p.sinfo[ki.sys];
    const int N = ki.nb, M = si.m, ld = N | 1, Np = tc_np(N);
    const bool live = 32 * q < Np;  // this warp holds rows of the padded matrix
    const float2* Hk = p.Hs + ki.offH;
    const double2* Hk64 = p.H + ki.offH;
    const double mu = p.mu[ki.sys];
    const double pib = M_PI / si.beta;
    for (int e = tid; e < M * N; e += blockDim.x) sP[e] = p.Ps[ki.offP + e];
    for (int x = tid; x < N; x += blockDim.x) sHii[x] = Hk64[x * N + x];
    __syncthreads();
    double acc_tr = 0.0, acc_g2 = 0.0;
    const uint32_t idesc = mma_idesc(2 * Np);

    for (int n = it.n0 + g; n < it.n1 && ok; n += NG) {
      const double wn = (2.0 * n + 1.0) * pib;
      for (int e = gt; e < M * M; e += 128) sS[e] = p.Ss[si.offSig + (int64_t)n * M * M + e];
      for (int x = gt; x < Np; x += 128)
        sD[x] = x < N ? make_float2(__double2float_rn(mu - sHii[x].x), __double2float_rn(wn - sHii[x].y))
                      : make_float2(1.f, 0.f);
      group_bar(1 + g);
      // T = Sigma P (M x Np, zero beyond N)
      for (int e = gt; e < M * Np; e += 128) {
        const int a = e / Np, j = e - a * Np;
        float2 acc = make_float2(0.f, 0.f);
        if (j < N)
          for (int b = 0; b < M; ++b) fmac(acc, sS[a * M + b], sP[b * N + j]);
        sT[e] = acc;
      }
      group_bar(1 + g);
      // A = diag - H - P^+ T, row i, written to tensor memory 8 columns at a time
      if (live) {
        for (int c0 = 0; c0 < Np; c0 += 8) {
          float re[8], im[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int c = c0 + j;
            float2 v = make_float2(0.f, 0.f);
            if (i < N && c < N) {
              const float2 h = Hk[(int64_t)i * N + c];
              v = (i == c) ? sD[i] : make_float2(-h.x, -h.y);
            } else if (i == c && i < Np) {
              v = sD[i];  // identity padding
            }
            re[j] = v.x;
            im[j] = v.y;
          }
          if (i < N) {
            for (int x = 0; x < M; ++x) {
              const float2 pv = sP[x * N + i];
              const float2 mp = make_float2(-pv.x, pv.y);  // -conj(P[x][i])
              const float4* t4 = reinterpret_cast<const float4*>(sT + x * Np + c0);
#pragma unroll
              for (int jj = 0; jj < 4; ++jj) {
                const float4 tt = t4[jj];
                re[2 * jj] = __fmaf_rn(mp.x, tt.x, __fmaf_rn(-mp.y, tt.y, re[2 * jj]));
                im[2 * jj] = __fmaf_rn(mp.x, tt.y, __fmaf_rn(mp.y, tt.x, im[2 * jj]));
                re[2 * jj + 1] = __fmaf_rn(mp.x, tt.z, __fmaf_rn(-mp.y, tt.w, re[2 * jj + 1]));
                im[2 * jj + 1] = __fmaf_rn(mp.x, tt.w, __fmaf_rn(mp.y, tt.z, im[2 * jj + 1]));
              }
            }
          }
          tmem_st8(tlane + (uint32_t)c0, re);
          tmem_st8(tlane + (uint32_t)(Np + c0), im);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      }

      unsigned used = 0u;  // this row was a pivot row
      int buf = 0;
      for (int j0 = 0; j0 < Np && ok; j0 += kTcB) {
        const int b = min(kTcB, Np - j0);  // 16, or 8 in a short last block
        // panel columns Q = [j0, j0 + b) of row i
        float vr[kTcB], vi[kTcB];
#pragma unroll
        for (int j = 0; j < kTcB; ++j) vr[j] = vi[j] = 0.f;
        if (live) {
          float t8[8];
          tmem_ld8(tlane + (uint32_t)j0, t8);
#pragma unroll
          for (int j = 0; j < 8; ++j) vr[j] = t8[j];
          tmem_ld8(tlane + (uint32_t)(Np + j0), t8);
#pragma unroll
          for (int j = 0; j < 8; ++j) vi[j] = t8[j];
          if (b == kTcB) {
            tmem_ld8(tlane + (uint32_t)(j0 + 8), t8);
#pragma unroll
            for (int j = 0; j < 8; ++j) vr[8 + j] = t8[j];
            tmem_ld8(tlane + (uint32_t)(Np + j0 + 8), t8);
#pragma unroll
            for (int j = 0; j < 8; ++j) vi[8 + j] = t8[j];
          }
        }
        int my_t = -1;  // pivot step of this row within the block
        if (b == kTcB)
          panel_sweep<kTcB>(vr, vi, used, my_t, i, Np, q, lane, g, gt, j0, buf, live, sStage, sKey, sPiv, p.status);
        else
          panel_sweep<8>(vr, vi, used, my_t, i, Np, q, lane, g, gt, j0, buf, live, sStage, sKey, sPiv, p.status);
        group_bar(1 + g);  // the block's pivot list is complete
        // B_op from the old pivot rows (tensor memory still holds them): row n < Np
        // carries output column c = n (real part), row Np + c its imaginary part.
        const unsigned own = live ? __ballot_sync(0xffffffffu, my_t >= 0) : 0u;
        if (own != 0u) {
          // the warp's pivot rows take slots 0 .. nown-1 in lane order
          const int nown = __popc(own), slot = __popc(own & ((1u << lane) - 1u));
          if (my_t >= 0) sSlotT[slot] = my_t;
          for (int c0 = 0; c0 < 2 * Np; c0 += 16) {
            float x16[16];
            tmem_ld16(tlane + (uint32_t)c0, x16);
            if (my_t >= 0) {  // owners of pivot rows stage their 16 values
              float4* w = reinterpret_cast<float4*>(sWst + slot * 16);
              w[0] = make_float4(x16[0], x16[1], x16[2], x16[3]);
              w[1] = make_float4(x16[4], x16[5], x16[6], x16[7]);
              w[2] = make_float4(x16[8], x16[9], x16[10], x16[11]);
              w[3] = make_float4(x16[12], x16[13], x16[14], x16[15]);
            }
            __syncwarp();
            for (int e = lane; e < nown * 16; e += 32) {
              const int sl = e >> 4, jj = e & 15;
              const int t = sSlotT[sl];
              const float val = sWst[sl * 16 + jj];
              const int col = c0 + jj;
              if (col < Np) {
                const int c = col;
                const float v = (c >= j0 && c < j0 + b) ? 0.f : val;
                put_split(bHi, bLo, op_off(c, t), v);
                put_split(bHi, bLo, op_off(Np + c, kTcB + t), v);
              } else {
                const int c = col - Np;
                const float v = (c >= j0 && c < j0 + b) ? 0.f : val;
                put_split(bHi, bLo, op_off(c, kTcB + t), -v);
                put_split(bHi, bLo, op_off(Np + c, t), v);
              }
            }
            __syncwarp();
          }
        }
        if (live) {
          // A_op row i: [Re L | Im L], L = new panel minus 1 at (p_t, t)
          float lr[kTcB], li[kTcB];
#pragma unroll
          for (int j = 0; j < kTcB; ++j) {
            const bool on = (i < Np) && (j < b);
            lr[j] = on ? vr[j] - ((j == my_t) ? 1.f : 0.f) : 0.f;
            li[j] = on ? vi[j] : 0.f;
          }
          // hi and lo TF32 parts of [Re L | Im L] into tensor memory (row i = lane i)
#pragma unroll
          for (int part = 0; part < 2; ++part) {
            const float* src = part ? li : lr;
            float h8[8], l8[8];
#pragma unroll
            for (int half = 0; half < 2; ++half) {
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const float x = src[8 * half + j];
                h8[j] = tf32_rna(x);
                l8[j] = tf32_rna(x - h8[j]);
              }
              const uint32_t col = acol + (uint32_t)(part * kTcB + 8 * half);
              tmem_st8(tlane + col, h8);
              tmem_st8(tlane + col + kTcK, l8);
            }
          }
          // the new panel columns into tensor memory (B_op is zero there, so the
          // GEMM leaves them)
          float t8[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) t8[j] = vr[j];
          tmem_st8(tlane + (uint32_t)j0, t8);
#pragma unroll
          for (int j = 0; j < 8; ++j) t8[j] = vi[j];
          tmem_st8(tlane + (uint32_t)(Np + j0), t8);
          if (b == kTcB) {
#pragma unroll
            for (int j = 0; j < 8; ++j) t8[j] = vr[8 + j];
            tmem_st8(tlane + (uint32_t)(j0 + 8), t8);
#pragma unroll
            for (int j = 0; j < 8; ++j) t8[j] = vi[8 + j];
            tmem_st8(tlane + (uint32_t)(Np + j0 + 8), t8);
          }
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        }
        proxy_fence();
        tc_fence_before();
        group_bar(1 + g);
        if (gt == 0 && !p.tc_skip_mma) {
          tc_fence_after();
          const uint32_t as[3] = {0u, 0u, (uint32_t)kTcK};  // hi, hi, lo
          const unsigned char* bs[3] = {bHi, bLo, bHi};
#pragma unroll
          for (int s = 0; s < 3; ++s)
#pragma unroll
            for (int kq = 0; kq < kTcK / 8; ++kq) {
              if (b < kTcB && (kq & 1)) continue;  // zero depth of a short block
              mma_tf32_ts(tmem, tmem + acol + as[s] + (uint32_t)(8 * kq),
                          smem_desc(smem_addr(bs[s]) + kq * 2 * kKChunk), idesc);
            }
          mma_commit(&s_bar[g]);
        }
        const bool done = mbar_wait(&s_bar[g], phase);
        phase ^= 1u;
        tc_fence_after();
        if (!__all_sync(0xffffffffu, done) && lane == 0) {
          atomicOr(p.status, kFlagTimeout);
          s_fail[g] = 1;
          s_abort = 1;
        }
        group_bar(1 + g);  // the group agrees on the outcome before its next block
        ok = (s_fail[g] == 0);
      }
      if (!ok) break;
      // X = B with rows and columns permuted: B to shared memory, then the traces
      if (live) {
        for (int c0 = 0; c0 < Np; c0 += 8) {
          float re[8], im[8];
          tmem_ld8(tlane + (uint32_t)c0, re);
          tmem_ld8(tlane + (uint32_t)(Np + c0), im);
          if (i < N) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
              if (c0 + j < N) sG[i * ld + c0 + j] = make_float2(re[j], im[j]);
          }
        }
      }
      // (a real column pivots on a padding row only when A is singular, which is
      // flagged; the clamp keeps the indices inside the stored rows)
      for (int j = gt; j < N; j += 128) sIdx[min(sPiv[j], N - 1)] = j;
      group_bar(1 + g);
      for (int x = gt; x < N; x += 128) sRow[x] = min(sPiv[x], N - 1) * ld;
      group_bar(1 + g);
      for (int x = gt; x < N; x += 128) acc_tr += (double)sG[sRow[x] + sIdx[x]].x;
      float g2 = 0.f;
      for (int e = gt; e < N * N; e += 128) {
        const int a = e / N, c = e - a * N;
        const float2 g1 = sG[sRow[a] + sIdx[c]], g3 = sG[sRow[c] + sIdx[a]];
        g2 = __fmaf_rn(g1.x, g3.x, __fmaf_rn(-g1.y, g3.y, g2));
      }
      acc_g2 += (double)g2;
      group_bar(1 + g);
    }
    const double tr_ = block_sum_tc(acc_tr, s_red);
    const double g2s = block_sum_tc(acc_g2, s_red);
    if (tid == 0) {
      double* o = p.occ_part + ((int64_t)kk * p.n_chunks + it.chunk) * 2;
      o[0] = tr_;
      o[1] = g2s;
    }
    __syncthreads();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem), "r"(acols));
  }
}

// Dynamic shared memory limit and the largest shared-memory carveout, so that the
// occupancy query and the launch see the same per-SM capacity.
template <int NG>
cudaError_t set_attrs_tc(size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(k_point_tc<NG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_point_tc<NG>, cudaFuncAttributePreferredSharedMemoryCarveout,
                              (int)cudaSharedmemCarveoutMaxShared);
}

template <int NG>
cudaError_t launch_tc(const PointParams& p, int grid, size_t smem, cudaStream_t s) {
  cudaError_t e = set_attrs_tc<NG>(smem);
  if (e != cudaSuccess) return e;
  k_point_tc<NG><<<grid, NG * 128, smem, s>>>(p);
  return cudaGetLastError();
}

template <int NG>
int bps_tc(size_t smem) {
  int nb = 0;
  if (set_attrs_tc<NG>(smem) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_point_tc<NG>, NG * 128, smem) != cudaSuccess) return 0;
  return nb;
}

}  // namespace

bool tc_fits(int nbmax, int ng) {
  return nbmax >= 1 && nbmax <= 128 && ng >= 1 && ng <= 4 && tc_alloc_cols(nbmax, ng) <= 512;
}

// Dynamic shared memory of a launch: the layout, raised where needed so that no
// more CTAs fit on an SM than its tensor memory holds (a CTA that cannot allocate
// would wait for another to exit).
size_t point_tc_smem(int nbmax, int mmax, int ng) {
  const size_t need = make_layout_tc(nbmax, mmax, ng).bytes;
  int dev = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess)
    return need;
  const int by_tmem = 512 / tc_alloc_cols(nbmax, ng);
  const size_t floor_bytes = (size_t)per_sm / (size_t)(by_tmem + 1) + 1;
  return need > floor_bytes ? need : floor_bytes;
}

// Resident CTAs per SM: the occupancy limit, and no more than the tensor memory
// (512 columns per SM) holds, since a CTA keeps its allocation for its lifetime.
int point_tc_blocks_per_sm(int nbmax, int ng, size_t smem) {
  int occ = 0;
  switch (ng) {
    case 1: occ = bps_tc<1>(smem); break;
    case 2: occ = bps_tc<2>(smem); break;
    case 3: occ = bps_tc<3>(smem); break;
    case 4: occ = bps_tc<4>(smem); break;
    default: return 0;
  }
  const int by_tmem = 512 / tc_alloc_cols(nbmax, ng);
  return occ < by_tmem ? occ : by_tmem;
}

cudaError_t launch_point_tc(int ng, const PointParams& p, int grid, size_t smem, cudaStream_t s) {
  switch (ng) {
    case 1: return launch_tc<1>(p, grid, smem, s);
    case 2: return launch_tc<2>(p, grid, smem, s);
    case 3: return launch_tc<3>(p, grid, smem, s);
    case 4: return launch_tc<4>(p, grid, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace gf
