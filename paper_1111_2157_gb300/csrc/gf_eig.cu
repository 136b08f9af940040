// Batched Hermitian eigensolver and the pole (pseudo-Hamiltonian) path (sm_103a).
//
// When Sigma has the pole form of Sec. 3.2.4 (Eq. se_pole),
//   Sigma(i w) = Sigma_inf + sum_i V_i^+ V_i / (i w - p_i),   V_i a 1 x m row,
// the band block of the resolvent of the pseudo-Hamiltonian of Sec. 3.3
// (Eq. pseudo_H_k), here with the pole energies shifted by mu,
//   H_ps = [[H_k + P^+ Sigma_inf P, W^+], [W, diag(p + mu)]],  W_i = V_i P_k,
// is G(k, i w_n) of Eq. dmftloop1 exactly.  With H_ps = Psi diag(E) Psi^+ the
// lattice sums follow in closed form (Eqs. rho_LDA+DMFT_componet_final, fix_mu):
//   rho_k = Psi_b diag(n_F(E - mu)) Psi_b^+,  N_k = sum_l |Psi_b,l|^2 n_F(E_l - mu),
//   G_loc(i w_n) = sum_k w_k sum_l phi_l phi_l^+ / (i w_n + mu - E_l),  phi_l = P Psi_b,l,
// where Psi_b is the band block (first N_b rows) of the eigenvectors.
//
// The eigensolver is the cyclic Jacobi method for complex Hermitian matrices
// with the round-robin (circle) ordering of disjoint pairs, so that one step
// applies N/2 independent rotations: one CTA per matrix, every thread on the
// column update, then on the row update, of its share of the pairs.  The
// matrix and the eigenvectors stay in shared memory when 2 N (N|1) 16-byte
// elements fit, else in a per-CTA slice of a global workspace (L2-resident).
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "gf_complex.cuh"
#include "gf_internal.cuh"

namespace gf {

namespace {

using namespace cx;

constexpr int kEigThreads = 256;


__device__ __forceinline__ double eig_block_sum(double v, double* red) {
  // Deterministic: fixed xor tree inside each warp, then warp 0 over the warps.
  for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double r = 0.0;
  for (int w = 0; w < kEigThreads / 32; ++w) r += red[w];
  __syncthreads();
  return r;  // the same value in every thread
}

// Fermi function n_F(x) = 1 / (e^{beta x} + 1) without overflow.
__device__ __forceinline__ double fermi(double x, double beta) {
  return 0.5 * (1.0 - tanh(0.5 * beta * x));
}

// Divided difference (n_F(x) - n_F(y)) / (x - y), n_F'(x) at x = y, from
// fx = n_F(x) and chx = cosh(beta x / 2): with u = beta (x - y) / 2 it is
// -(beta/4) (sinh u / u) / (cosh(beta x/2) cosh(beta y/2)) (tanh difference
// formula), used for |u| <= 1 where the plain quotient would cancel; an
// infinite cosh gives the correct limit 0.  For |u| > 1 the plain quotient
// loses at most 2^-52 / |x - y| <= 2^-53 beta in absolute terms.
__device__ __forceinline__ double fermi_divdiff(double x, double y, double fx, double fy,
                                                double chx, double chy, double beta) {
  const double u = 0.5 * beta * (x - y);
  if (fabs(u) > 1.0) return (fx - fy) / (x - y);
  const double su = fabs(u) < 1e-4 ? fma(u * u, 1.0 / 6.0, 1.0) : sinh(u) / u;
  return -0.25 * beta * su / (chx * chy);
}

// Pair k of round-robin step r over np2 (even) indices: the last index stays,
// the others rotate.  Every unordered pair occurs once in np2 - 1 steps.
__device__ __forceinline__ void rr_pair(int r, int k, int np2, int& p, int& q) {
  const int m = np2 - 1;
  int a, b;
  if (k == 0) {
    a = m;
    b = r;
  } else {
    a = (r + k) % m;
    b = (r - k + m) % m;
  }
  p = min(a, b);
  q = max(a, b);
}

// Cyclic Jacobi on the Hermitian N x N matrix A (row-major, leading dimension
// ld, full storage); V receives the eigenvectors as columns (V = I on entry is
// set here).  On return the diagonal of A holds the eigenvalues.  Scratch:
// rot[4 * npair] doubles and ph[npair] complex in shared memory.  Returns the
// number of sweeps, or -1 when max_sweeps did not reach the threshold
// off(A) <= 1e-30 ||A||_F^2.
__device__ int jacobi_heev(double2* A, double2* V, int N, int ld, int max_sweeps, double* rot,
                           double2* ph, double* red) {
  const int tid = threadIdx.x;
  for (int e = tid; e < N * N; e += kEigThreads) {
    const int i = e / N, j = e - (e / N) * N;
    V[i * ld + j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  const int np2 = N + (N & 1);
  const int npair = np2 / 2;
  __syncthreads();
  for (int sweep = 0;; ++sweep) {
    double off = 0.0, all = 0.0;
    for (int e = tid; e < N * N; e += kEigThreads) {
      const int i = e / N, j = e - (e / N) * N;
      const double2 a = A[i * ld + j];
      const double s = a.x * a.x + a.y * a.y;
      all += s;
      if (i != j) off += s;
    }
    off = eig_block_sum(off, red);
    all = eig_block_sum(all, red);
    if (off <= 1e-30 * all || off == 0.0) return sweep;
    if (sweep >= max_sweeps) return -1;
    for (int r = 0; r < np2 - 1; ++r) {
      // rotation of each pair: J = [[c, s], [-s e, c e]] with e = conj(b)/|b|
      for (int k = tid; k < npair; k += kEigThreads) {
        int p, q;
        rr_pair(r, k, np2, p, q);
        double c = 1.0, s = 0.0, dp = 0.0, dq = 0.0;
        double2 e = make_double2(1.0, 0.0);
        if (q < N) {
          const double2 b = A[p * ld + q];
          const double ab = hypot(b.x, b.y);
          const double a = A[p * ld + p].x, d = A[q * ld + q].x;
          if (ab > 0.0) {
            const double zeta = (d - a) / (2.0 * ab);
            const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
            c = 1.0 / sqrt(fma(t, t, 1.0));
            s = t * c;
            e = make_double2(b.x / ab, -b.y / ab);
            dp = a - t * ab;
            dq = d + t * ab;
          } else {
            dp = a;
            dq = d;
          }
        }
        rot[4 * k + 0] = c;
        rot[4 * k + 1] = s;
        rot[4 * k + 2] = dp;
        rot[4 * k + 3] = dq;
        ph[k] = e;
      }
      __syncthreads();
      // columns: M[:, p] <- c M[:, p] - s e M[:, q];  M[:, q] <- s M[:, p] + c e M[:, q]
      for (int x = tid; x < 2 * N * npair; x += kEigThreads) {
        const int which = x >= N * npair;  // 0: A, 1: V
        const int y = x - which * N * npair;
        const int k = y / N, i = y - (y / N) * N;
        int p, q;
        rr_pair(r, k, np2, p, q);
        if (q >= N) continue;
        const double c = rot[4 * k + 0], s = rot[4 * k + 1];
        if (s == 0.0 && ph[k].x == 1.0 && ph[k].y == 0.0) continue;
        double2* M = which ? V : A;
        const double2 xp = M[i * ld + p], xq = M[i * ld + q];
        const double2 eq = cmul(ph[k], xq);
        M[i * ld + p] = make_double2(c * xp.x - s * eq.x, c * xp.y - s * eq.y);
        M[i * ld + q] = make_double2(s * xp.x + c * eq.x, s * xp.y + c * eq.y);
      }
      __syncthreads();
      // rows of A: A[p, :] <- c A[p, :] - s conj(e) A[q, :];  A[q, :] <- s A[p, :] + c conj(e) A[q, :]
      for (int y = tid; y < N * npair; y += kEigThreads) {
        const int k = y / N, j = y - (y / N) * N;
        int p, q;
        rr_pair(r, k, np2, p, q);
        if (q >= N) continue;
        const double c = rot[4 * k + 0], s = rot[4 * k + 1];
        if (j == p) {
          A[p * ld + p] = make_double2(rot[4 * k + 2], 0.0);
          A[q * ld + p] = make_double2(0.0, 0.0);
          continue;
        }
        if (j == q) {
          A[q * ld + q] = make_double2(rot[4 * k + 3], 0.0);
          A[p * ld + q] = make_double2(0.0, 0.0);
          continue;
        }
        if (s == 0.0 && ph[k].x == 1.0 && ph[k].y == 0.0) continue;
        const double2 ec = make_double2(ph[k].x, -ph[k].y);
        const double2 xp = A[p * ld + j], xq = A[q * ld + j];
        const double2 eq = cmul(ec, xq);
        A[p * ld + j] = make_double2(c * xp.x - s * eq.x, c * xp.y - s * eq.y);
        A[q * ld + j] = make_double2(s * xp.x + c * eq.x, s * xp.y + c * eq.y);
      }
      __syncthreads();
    }
  }
}

__device__ __forceinline__ size_t eig_ws_elems(int n) { return (size_t)2 * n * (n | 1); }

// Standalone batched eigensolver: A [mat][n][n] -> w [mat][n] ascending,
// V [mat][n][n] with eigenvector l in column l.
__global__ void __launch_bounds__(kEigThreads)
    k_heev_batched(const double2* __restrict__ Ain, int n_mat, int n, int max_sweeps,
                   double* __restrict__ w_out, double2* __restrict__ v_out, double2* gws,
                   int in_smem, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double rot[4 * 128];
  __shared__ double2 ph[128];
  __shared__ double red[kEigThreads / 32];
  const int ld = n | 1;
  double2* A = in_smem ? reinterpret_cast<double2*>(smem_raw) : gws + blockIdx.x * eig_ws_elems(n);
  double2* V = A + (size_t)n * ld;
  for (int mat = blockIdx.x; mat < n_mat; mat += gridDim.x) {
    const double2* src = Ain + (size_t)mat * n * n;
    for (int e = threadIdx.x; e < n * n; e += kEigThreads) {
      const int i = e / n, j = e - (e / n) * n;
      // Hermitian part of the input: (A + A^+)/2
      const double2 a = src[i * n + j], b = src[j * n + i];
      A[i * ld + j] = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
    }
    __syncthreads();
    const int sw = jacobi_heev(A, V, n, ld, max_sweeps, rot, ph, red);
    if (sw < 0 && threadIdx.x == 0) atomicOr(status, 2);
    // ascending order; equal values keep their index order
    for (int i = threadIdx.x; i < n; i += kEigThreads) {
      const double li = A[i * ld + i].x;
      int rank = 0;
      for (int j = 0; j < n; ++j) {
        const double lj = A[j * ld + j].x;
        rank += (lj < li) || (lj == li && j < i);
      }
      w_out[(size_t)mat * n + rank] = li;
      for (int r = 0; r < n; ++r) v_out[(size_t)mat * n * n + (size_t)r * n + rank] = V[r * ld + i];
    }
    __syncthreads();
  }
}

// Pole path, one CTA per k (grid-stride over k): build H_ps(mu), diagonalise,
// and reduce in the epilogue selected by mode:
//   kOcc:  kN[k] = sum_l |Psi_b,l|^2 n_F(E_l - mu),
//          kdN[k] = dN_k/dmu = -sum_{l,l'} |(Psi_b^+ Psi_b)_{l l'}|^2 n_F[1](E_l - mu, E_l' - mu)
//          (the derivative of Tr[Pi_b n_F(H_0 - mu Pi_b)] with the pole block of
//          H_0 unshifted; n_F[1] is the divided difference);
//   kRho:  rho_k = Psi_b diag(n_F) Psi_b^+ and kNc[k] = sum_l |phi_l|^2 n_F;
//   kGloc: E_l and phi_l = P Psi_b,l to eout / phiout for k_pole_gloc.
__global__ void __launch_bounds__(kEigThreads) k_pole_eig(const PoleParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double s_x[256], s_f[256], s_ch[256];
  __shared__ double rot[4 * 128];
  __shared__ double2 ph[128];
  __shared__ double red[kEigThreads / 32];
  const int tid = threadIdx.x;
  for (int k = blockIdx.x; k < p.n_k; k += gridDim.x) {
    const KInfo ki = p.kinfo[k];
    const SInfo si = p.sinfo[ki.sys];
    const PInfo pi = p.pinfo[ki.sys];
    const int nb = ki.nb, m = si.m, npl = pi.np, n = nb + npl, ld = n | 1;
    const double mu = p.mu[ki.sys];
    double2* A = p.in_smem ? reinterpret_cast<double2*>(smem_raw) : p.ws + blockIdx.x * p.ws_stride;
    double2* V = A + (size_t)n * ld;
    const double2* H = p.H + ki.offH;
    const double2* P = p.P + ki.offP;
    const double2* Sinf = p.Sinf + si.offSinf;
    const double2* Vp = p.Vp + pi.offV;
    double2* Vs = p.vstore ? p.vstore + p.voff[k] : nullptr;  // eigenvectors kept between calls
    double* Es = p.estore ? p.estore + p.eoff[k] : nullptr;
    if (p.warm) {
      // warm start from the eigenpairs (E', V') at mu' = mu_prev: H_ps(mu) = H_ps(mu') +
      // (mu - mu') Pi_p, so V'^+ H_ps(mu) V' = diag(E') + (mu - mu') V_p'^+ V_p' with V_p'
      // the pole rows of V'; Jacobi then only removes what the shift of mu added
      const double dmu = mu - p.mu_prev[ki.sys];
      for (int e = tid; e < n * n; e += kEigThreads) {
        const int l = e / n, l2 = e - (e / n) * n;
        double2 acc = make_double2(0.0, 0.0);
        for (int i = nb; i < n; ++i) cmac_ca(acc, Vs[i * n + l], Vs[i * n + l2]);
        acc.x *= dmu;
        acc.y *= dmu;
        if (l == l2) acc.x += Es[l];
        A[l * ld + l2] = acc;
      }
    } else {
      // band block H + P^+ Sigma_inf P
      for (int e = tid; e < nb * nb; e += kEigThreads) {
        const int i = e / nb, j = e - (e / nb) * nb;
        double2 acc = H[i * nb + j];
        for (int a = 0; a < m; ++a) {
          double2 t = make_double2(0.0, 0.0);
          for (int b = 0; b < m; ++b) cmac(t, Sinf[a * m + b], P[b * nb + j]);
          cmac_ca(acc, P[a * nb + i], t);
        }
        A[i * ld + j] = acc;
      }
      // pole rows/columns W_i = V_i P and the pole diagonal p_i + mu
      for (int e = tid; e < npl * nb; e += kEigThreads) {
        const int i = e / nb, b = e - (e / nb) * nb;
        double2 w = make_double2(0.0, 0.0);
        for (int a = 0; a < m; ++a) cmac(w, Vp[i * m + a], P[a * nb + b]);
        A[(nb + i) * ld + b] = w;
        A[b * ld + nb + i] = make_double2(w.x, -w.y);
      }
      for (int e = tid; e < npl * npl; e += kEigThreads) {
        const int i = e / npl, j = e - (e / npl) * npl;
        A[(nb + i) * ld + nb + j] = make_double2(i == j ? p.poles[pi.offp + i] + mu : 0.0, 0.0);
      }
    }
    __syncthreads();
    const int sw = jacobi_heev(A, V, n, ld, p.max_sweeps, rot, ph, red);
    if (sw < 0 && tid == 0) atomicOr(p.status, 2);
    if (p.warm) {
      // eigenvectors of H_ps(mu) = V' R: the product goes to A's storage (its
      // diagonal, the eigenvalues, is kept in s_x first) and A, V swap roles
      for (int l = tid; l < n; l += kEigThreads) s_x[l] = A[l * ld + l].x;
      __syncthreads();
      for (int e = tid; e < n * n; e += kEigThreads) {
        const int i = e / n, l = e - (e / n) * n;
        double2 acc = make_double2(0.0, 0.0);
        for (int q = 0; q < n; ++q) cmac(acc, Vs[i * n + q], V[q * ld + l]);
        A[i * ld + l] = acc;
      }
      __syncthreads();
      double2* t = A;
      A = V;
      V = t;
      for (int l = tid; l < n; l += kEigThreads) A[l * ld + l] = make_double2(s_x[l], 0.0);
      __syncthreads();
    }
    if (p.save_v) {
      for (int e = tid; e < n * n; e += kEigThreads) {
        const int i = e / n, l = e - (e / n) * n;
        Vs[e] = V[i * ld + l];
      }
      for (int l = tid; l < n; l += kEigThreads) Es[l] = A[l * ld + l].x;
    }
    // per eigenpair: x_l = E_l - mu, n_F(x_l), cosh(beta x_l / 2)
    for (int l = tid; l < n; l += kEigThreads) {
      const double x = A[l * ld + l].x - mu;
      s_x[l] = x;
      s_f[l] = fermi(x, si.beta);
      s_ch[l] = cosh(0.5 * si.beta * x);
    }
    __syncthreads();
    if (p.mode & kOcc) {
      double nk = 0.0;
      for (int l = tid; l < n; l += kEigThreads) {
        double wb = 0.0;
        for (int b = 0; b < nb; ++b) {
          const double2 v = V[b * ld + l];
          wb = fma(v.x, v.x, fma(v.y, v.y, wb));
        }
        nk = fma(wb, s_f[l], nk);
      }
      nk = eig_block_sum(nk, red);
      double dk = 0.0;
      for (int e = tid; e < n * n; e += kEigThreads) {
        const int l = e / n, l2 = e - (e / n) * n;
        double2 o = make_double2(0.0, 0.0);
        for (int b = 0; b < nb; ++b) cmac_ca(o, V[b * ld + l], V[b * ld + l2]);
        const double f1 =
            fermi_divdiff(s_x[l], s_x[l2], s_f[l], s_f[l2], s_ch[l], s_ch[l2], si.beta);
        dk = fma(-(o.x * o.x + o.y * o.y), f1, dk);
      }
      dk = eig_block_sum(dk, red);
      if (tid == 0) {
        p.kN[k] = nk;
        p.kdN[k] = dk;
      }
    }
    if (p.mode & kRho) {
      double2* rho = p.rho + ki.offH;
      double hks = 0.0;  // Re Tr(H_k rho_k)
      for (int e = tid; e < nb * nb; e += kEigThreads) {
        const int i = e / nb, j = e - (e / nb) * nb;
        double2 acc = make_double2(0.0, 0.0);
        for (int l = 0; l < n; ++l) {
          const double f = s_f[l];
          double2 vi = V[i * ld + l];
          vi.x *= f;
          vi.y *= f;
          cmac_cb(acc, vi, V[j * ld + l]);
        }
        rho[i * nb + j] = acc;
        const double2 h = H[j * nb + i];
        hks = fma(h.x, acc.x, fma(-h.y, acc.y, hks));
      }
      double nc = 0.0;
      for (int e = tid; e < m * n; e += kEigThreads) {
        const int a = e / n, l = e - (e / n) * n;
        double2 f = make_double2(0.0, 0.0);
        for (int b = 0; b < nb; ++b) cmac(f, P[a * nb + b], V[b * ld + l]);
        nc = fma(f.x * f.x + f.y * f.y, s_f[l], nc);
      }
      // sum_l (E_l - mu) |Psi_b,l|^2 n_F(E_l - mu)
      double eps = 0.0;
      for (int l = tid; l < n; l += kEigThreads) {
        double wb = 0.0;
        for (int b = 0; b < nb; ++b) {
          const double2 v = V[b * ld + l];
          wb = fma(v.x, v.x, fma(v.y, v.y, wb));
        }
        eps = fma(s_x[l] * wb, s_f[l], eps);
      }
      nc = eig_block_sum(nc, red);
      hks = eig_block_sum(hks, red);
      eps = eig_block_sum(eps, red);
      if (tid == 0) {
        p.kNc[k] = nc;
        if (p.kHks) p.kHks[k] = hks;
        if (p.kEps) p.kEps[k] = eps;
      }
    }
    if (p.mode & kGloc) {
      double* E = p.eout + p.eoff[k];
      double2* phi = p.phiout + p.phioff[k];
      for (int l = tid; l < n; l += kEigThreads) {
        E[l] = A[l * ld + l].x;
        if (p.wbout) {
          double wb = 0.0;
          for (int b = 0; b < nb; ++b) {
            const double2 v = V[b * ld + l];
            wb = fma(v.x, v.x, fma(v.y, v.y, wb));
          }
          p.wbout[p.eoff[k] + l] = wb;
        }
      }
      for (int e = tid; e < m * n; e += kEigThreads) {
        const int a = e / n, l = e - (e / n) * n;
        double2 f = make_double2(0.0, 0.0);
        for (int b = 0; b < nb; ++b) cmac(f, P[a * nb + b], V[b * ld + l]);
        phi[a * n + l] = f;
      }
    }
    __syncthreads();
  }
}

// G_loc(i w_n) = sum_k w_k sum_l phi_l phi_l^+ / (i w_n + mu - E_l) for one
// system and F consecutive frequencies per CTA.  With t = phi_a conj(phi_b)
// and g = w_k / (i w + mu - E) = gr + i gi: G_ab = Xr + i Xi and
// G_ba = conj(Xr) + i conj(Xi) with Xr = sum t gr, Xi = sum t gi, so each
// thread sums QP pairs a <= b.  phi and E are staged in shared memory kCh
// eigenpairs at a time; the sums run over k, then l, in increasing order.
constexpr int kCh = 32;

template <int QP, int F>
__global__ void __launch_bounds__(kEigThreads)
    k_pole_gloc(const PoleParams p, int blocks_per_sys, int n_split, double2* part, int64_t tot) {
  __shared__ double2 s_phi[32 * kCh];  // m <= 32
  __shared__ double2 s_g[F * kCh];
  const int s = blockIdx.x / blocks_per_sys;
  const int f0 = (blockIdx.x - s * blocks_per_sys) * F;
  const int split = blockIdx.y;
  const SInfo si = p.sinfo[s];
  // k-points [ka, kb) of this split of the system
  const int nks = si.k1 - si.k0;
  const int ka = si.k0 + (int)((int64_t)nks * split / n_split);
  const int kb = si.k0 + (int)((int64_t)nks * (split + 1) / n_split);
  const int m = si.m;
  const int npairs = m * (m + 1) / 2;
  const double mu = p.mu[s];
  const int tid = threadIdx.x;
  int pa[QP], pb[QP];
#pragma unroll
  for (int q = 0; q < QP; ++q) {
    int rem = tid + q * kEigThreads, a = 0;
    if (rem >= npairs) rem = 0;
    while (rem >= m - a) { rem -= m - a; ++a; }
    pa[q] = a;
    pb[q] = a + rem;
  }
  double2 xr[QP][F], xi[QP][F];
#pragma unroll
  for (int q = 0; q < QP; ++q)
#pragma unroll
    for (int f = 0; f < F; ++f) {
      xr[q][f] = make_double2(0.0, 0.0);
      xi[q][f] = make_double2(0.0, 0.0);
    }
  for (int k = ka; k < kb; ++k) {
    const int n = p.kinfo[k].nb + p.pinfo[s].np;
    const double wk = p.kinfo[k].w;
    const double* E = p.eout + p.eoff[k];
    const double2* phi = p.phiout + p.phioff[k];
    for (int l0 = 0; l0 < n; l0 += kCh) {
      const int cl = min(kCh, n - l0);
      __syncthreads();
      for (int e = tid; e < m * cl; e += kEigThreads) {
        const int a = e / cl, l = e - (e / cl) * cl;
        s_phi[a * kCh + l] = phi[a * n + l0 + l];
      }
      for (int e = tid; e < F * cl; e += kEigThreads) {
        const int f = e / cl, l = e - (e / cl) * cl;
        const int nn = f0 + f;
        const double wn = (2.0 * nn + 1.0) * 3.14159265358979323846 / si.beta;
        // w_k / (mu - E + i w) = w_k (x - i w) / (x^2 + w^2), x = mu - E
        const double x = mu - E[l0 + l];
        const double d = wk / fma(x, x, wn * wn);
        s_g[f * kCh + l] = make_double2(x * d, -wn * d);
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < QP; ++q) {
        if (tid + q * kEigThreads >= npairs) continue;
        const int a = pa[q], b = pb[q];
        for (int l = 0; l < cl; ++l) {
          double2 t = make_double2(0.0, 0.0);
          cmac_cb(t, s_phi[a * kCh + l], s_phi[b * kCh + l]);
#pragma unroll
          for (int f = 0; f < F; ++f) {
            const double2 g = s_g[f * kCh + l];
            xr[q][f].x = fma(t.x, g.x, xr[q][f].x);
            xr[q][f].y = fma(t.y, g.x, xr[q][f].y);
            xi[q][f].x = fma(t.x, g.y, xi[q][f].x);
            xi[q][f].y = fma(t.y, g.y, xi[q][f].y);
          }
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < QP; ++q) {
    if (tid + q * kEigThreads >= npairs) continue;
    const int a = pa[q], b = pb[q];
#pragma unroll
    for (int f = 0; f < F; ++f) {
      const int nn = f0 + f;
      if (nn >= p.n_iw) continue;
      double2* out = part + (int64_t)split * tot + si.offSig + (int64_t)nn * m * m;
      out[a * m + b] = make_double2(xr[q][f].x - xi[q][f].y, xr[q][f].y + xi[q][f].x);
      out[b * m + a] = make_double2(xr[q][f].x + xi[q][f].y, xi[q][f].x - xr[q][f].y);
    }
  }
}

// gloc[e] = sum over the splits, in order, of part[split][e].
__global__ void k_split_reduce(const double2* __restrict__ part, int n_split, int64_t tot,
                               double2* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    double2 acc = part[e];
    for (int sp = 1; sp < n_split; ++sp) {
      const double2 v = part[(int64_t)sp * tot + e];
      acc.x += v.x;
      acc.y += v.y;
    }
    out[e] = acc;
  }
}

// Low-rank path setup, one CTA per k (grid-stride): H_k = U diag(eps) U^+ by
// Jacobi, then Pt = P_k U.
__global__ void __launch_bounds__(kEigThreads)
    k_lr_setup(const double2* __restrict__ H, const double2* __restrict__ P,
               const KInfo* __restrict__ kinfo, const SInfo* __restrict__ sinfo,
               const int64_t* __restrict__ offD, int n_k, int nbmax, double* __restrict__ eps,
               double2* __restrict__ U, double2* __restrict__ Pt, double2* gws, int in_smem,
               int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double rot[4 * 128];
  __shared__ double2 ph[128];
  __shared__ double red[kEigThreads / 32];
  double2* A = in_smem ? reinterpret_cast<double2*>(smem_raw) : gws + blockIdx.x * eig_ws_elems(nbmax);
  for (int k = blockIdx.x; k < n_k; k += gridDim.x) {
    const KInfo ki = kinfo[k];
    const int n = ki.nb, m = sinfo[ki.sys].m, ld = n | 1;
    double2* V = A + (size_t)n * ld;
    const double2* Hk = H + ki.offH;
    for (int e = threadIdx.x; e < n * n; e += kEigThreads) {
      const int i = e / n, j = e - (e / n) * n;
      const double2 a = Hk[i * n + j], b = Hk[j * n + i];
      A[i * ld + j] = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
    }
    __syncthreads();
    const int sw = jacobi_heev(A, V, n, ld, 40, rot, ph, red);
    if (sw < 0 && threadIdx.x == 0) atomicOr(status, 2);
    for (int l = threadIdx.x; l < n; l += kEigThreads) eps[offD[k] + l] = A[l * ld + l].x;
    for (int e = threadIdx.x; e < n * n; e += kEigThreads) {
      const int i = e / n, l = e - (e / n) * n;
      U[ki.offH + e] = V[i * ld + l];
    }
    const double2* Pk = P + ki.offP;
    for (int e = threadIdx.x; e < m * n; e += kEigThreads) {
      const int a = e / n, l = e - (e / n) * n;
      double2 acc = make_double2(0.0, 0.0);
      for (int b = 0; b < n; ++b) cmac(acc, Pk[a * n + b], V[b * ld + l]);
      Pt[ki.offP + e] = acc;
    }
    __syncthreads();
  }
}

// DOS and PDOS on the real axis from the pseudo-Hamiltonian eigenpairs
// (Eqs. DOS and PDOS) with a Lorentzian of half width eta:
//   D(e)       = sum_k w_k sum_l |Psi_b,l|^2 L(e + mu - E_l),
//   D_alpha(e) = sum_k w_k sum_l |phi_l(alpha)|^2 L(e + mu - E_l),
//   L(x) = (eta / pi) / (x^2 + eta^2) = -(1/pi) Im 1/(x + i eta).
// One thread per (system, energy); the k and l sums run in increasing order.
__global__ void k_pole_dos(const PoleParams p, const double* __restrict__ eps_grid, int n_eps,
                           double eta, const int64_t* __restrict__ pdos_off, double* __restrict__ dos,
                           double* __restrict__ pdos) {
  const int s = blockIdx.y;
  const int ie = blockIdx.x * blockDim.x + threadIdx.x;
  if (ie >= n_eps) return;
  const SInfo si = p.sinfo[s];
  const int m = si.m, npl = p.pinfo[s].np;
  const double z = eps_grid[ie] + p.mu[s];
  double d = 0.0;
  double pd[32];
  for (int a = 0; a < 32; ++a) pd[a] = 0.0;
  for (int k = si.k0; k < si.k1; ++k) {
    const int n = p.kinfo[k].nb + npl;
    const double wk = p.kinfo[k].w;
    const double* E = p.eout + p.eoff[k];
    const double* wb = p.wbout + p.eoff[k];
    const double2* phi = p.phiout + p.phioff[k];
    for (int l = 0; l < n; ++l) {
      const double x = z - E[l];
      const double lor = wk * (eta * 0.31830988618379067) / fma(x, x, eta * eta);
      d = fma(wb[l], lor, d);
      if (pdos)
        for (int a = 0; a < m; ++a) {
          const double2 f = phi[a * n + l];
          pd[a] = fma(fma(f.x, f.x, f.y * f.y), lor, pd[a]);
        }
    }
  }
  dos[(int64_t)s * n_eps + ie] = d;
  if (pdos)
    for (int a = 0; a < m; ++a) pdos[pdos_off[s] + (int64_t)ie * m + a] = pd[a];
}

// Orthonormal projectors of Eqs. 6 and 7 (Lowdin):
// P_k = O^{-1/2} W_k, O = W_k W_k^+ (m x m), one CTA per k.  O's eigenpairs by
// the Jacobi routine; eigenvalues <= tol * max eigenvalue flag the k-point
// (linearly dependent projections).
__global__ void __launch_bounds__(kEigThreads)
    k_lowdin(const KInfo* __restrict__ kinfo, const SInfo* __restrict__ sinfo,
             const double2* __restrict__ Wraw, double2* __restrict__ Pout, int mmax, int* status) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double rot[4 * 16];
  __shared__ double2 ph[16];
  __shared__ double red[kEigThreads / 32];
  __shared__ double s_isq[32];
  const int k = blockIdx.x;
  const KInfo ki = kinfo[k];
  const int N = ki.nb, M = sinfo[ki.sys].m, ld = M | 1;
  double2* O = reinterpret_cast<double2*>(smraw);
  double2* V = O + M * ld;
  double2* T = V + M * ld;  // O^{-1/2}
  const double2* Wk = Wraw + ki.offP;
  for (int e = threadIdx.x; e < M * M; e += kEigThreads) {
    const int a = e / M, b = e - (e / M) * M;
    double2 acc = make_double2(0.0, 0.0);
    for (int j = 0; j < N; ++j) cmac_cb(acc, Wk[a * N + j], Wk[b * N + j]);
    O[a * ld + b] = acc;
  }
  __syncthreads();
  const int sw = jacobi_heev(O, V, M, ld, 40, rot, ph, red);
  if (sw < 0 && threadIdx.x == 0) atomicOr(status, 2);
  if (threadIdx.x == 0) {
    double lmax = 0.0;
    for (int l = 0; l < M; ++l) lmax = fmax(lmax, O[l * ld + l].x);
    for (int l = 0; l < M; ++l) {
      const double lam = O[l * ld + l].x;
      if (!(lam > 1e-12 * lmax)) {
        atomicOr(status, kFlagSingular);
        s_isq[l] = 0.0;
      } else {
        s_isq[l] = 1.0 / sqrt(lam);
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < M * M; e += kEigThreads) {
    const int a = e / M, b = e - (e / M) * M;
    double2 acc = make_double2(0.0, 0.0);
    for (int l = 0; l < M; ++l) {
      double2 v = V[a * ld + l];
      v.x *= s_isq[l];
      v.y *= s_isq[l];
      cmac_cb(acc, v, V[b * ld + l]);
    }
    T[a * ld + b] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < M * N; e += kEigThreads) {
    const int a = e / N, j = e - (e / N) * N;
    double2 acc = make_double2(0.0, 0.0);
    for (int b = 0; b < M; ++b) cmac(acc, T[a * ld + b], Wk[b * N + j]);
    Pout[ki.offP + e] = acc;
  }
}

}  // namespace

cudaError_t launch_lr_setup(const double2* H, const double2* P, const KInfo* kinfo,
                            const SInfo* sinfo, const int64_t* offD, int n_k, int nbmax,
                            double* eps, double2* U, double2* Pt, double2* ws, int grid,
                            int in_smem, int* status, cudaStream_t s) {
  const size_t smem = in_smem ? heev_smem(nbmax) : 0;
  cudaError_t e =
      cudaFuncSetAttribute(k_lr_setup, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_lr_setup<<<grid, kEigThreads, smem, s>>>(H, P, kinfo, sinfo, offD, n_k, nbmax, eps, U, Pt, ws,
                                             in_smem, status);
  return cudaGetLastError();
}

cudaError_t launch_lowdin(const KInfo* kinfo, const SInfo* sinfo, int n_k, int mmax,
                          const double2* Wraw, double2* Pout, int* status, cudaStream_t s) {
  const size_t smem = (size_t)3 * mmax * (mmax | 1) * sizeof(double2);
  cudaError_t e = cudaFuncSetAttribute(k_lowdin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_lowdin<<<n_k, kEigThreads, smem, s>>>(kinfo, sinfo, Wraw, Pout, mmax, status);
  return cudaGetLastError();
}

cudaError_t launch_pole_dos(const PoleParams& p, int n_sys, const double* eps_grid, int n_eps,
                            double eta, const int64_t* pdos_off, double* dos, double* pdos,
                            cudaStream_t s) {
  dim3 grid((n_eps + 127) / 128, n_sys);
  k_pole_dos<<<grid, 128, 0, s>>>(p, eps_grid, n_eps, eta, pdos_off, dos, pdos);
  return cudaGetLastError();
}

size_t heev_smem(int n) { return (size_t)2 * n * (n | 1) * sizeof(double2); }
size_t heev_ws_elems(int n) { return (size_t)2 * n * (n | 1); }
int heev_max_n() { return 2 * 128; }  // rotation scratch holds 128 pairs

cudaError_t launch_heev_batched(const double2* A, int n_mat, int n, int max_sweeps, double* w,
                                double2* V, double2* gws, int grid, int in_smem, int* status,
                                cudaStream_t s) {
  const size_t smem = in_smem ? heev_smem(n) : 0;
  cudaError_t e = cudaFuncSetAttribute(k_heev_batched, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_heev_batched<<<grid, kEigThreads, smem, s>>>(A, n_mat, n, max_sweeps, w, V, gws, in_smem, status);
  return cudaGetLastError();
}

cudaError_t launch_pole_eig(const PoleParams& p, int grid, size_t smem, cudaStream_t s) {
  cudaError_t e =
      cudaFuncSetAttribute(k_pole_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_pole_eig<<<grid, kEigThreads, smem, s>>>(p);
  return cudaGetLastError();
}

// frequencies per CTA of k_pole_gloc: 8 with one pair per thread, else 4
int pole_gloc_f(int mmax) { return mmax * (mmax + 1) / 2 <= kEigThreads ? 8 : 4; }

int pole_gloc_splits(int n_sys, int n_iw, int sm_count, int mmax) {
  const int F = pole_gloc_f(mmax);
  const int blocks = n_sys * ((n_iw + F - 1) / F);
  return std::max(1, std::min(64, (2 * sm_count + blocks - 1) / blocks));
}

cudaError_t launch_pole_gloc(const PoleParams& p, int n_sys, int mmax, int n_split, double2* part,
                             int64_t tot, cudaStream_t s) {
  const int F = pole_gloc_f(mmax);
  const int bps = (p.n_iw + F - 1) / F;
  const dim3 grid(n_sys * bps, n_split);
  const int qp = (mmax * (mmax + 1) / 2 + kEigThreads - 1) / kEigThreads;  // 1..3 for m <= 32
  if (qp <= 1) k_pole_gloc<1, 8><<<grid, kEigThreads, 0, s>>>(p, bps, n_split, part, tot);
  else if (qp <= 2) k_pole_gloc<2, 4><<<grid, kEigThreads, 0, s>>>(p, bps, n_split, part, tot);
  else k_pole_gloc<3, 4><<<grid, kEigThreads, 0, s>>>(p, bps, n_split, part, tot);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_split_reduce<<<std::min<int64_t>(4096, (tot + 255) / 256), 256, 0, s>>>(part, n_split, tot, p.gloc);
  return cudaGetLastError();
}

}  // namespace gf
