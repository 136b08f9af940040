// C-ABI of libgf, continued: the pole (pseudo-Hamiltonian) path, the batched
// eigensolver, the projector orthonormalisation and the DMFT-step entry points.
#include "gf_ctx.cuh"

namespace {

// Pole path: build H_ps(mu) per k, diagonalise, and run the epilogues of mode.
gf_status pole_run(gf_ctx* c, int mode, bool gloc_kernel = true, int warm = 0, int save_v = 0) {
  if (!c->have_H || !c->have_P || !c->have_poles)
    return fail(c, GF_ESTATE, "gf_set_hamiltonian, gf_set_projectors and gf_set_sigma_poles must "
                              "all be called before a pole-path call");
  GF_CU(cudaMemsetAsync(c->status.p, 0, sizeof(int), c->stream));
  gf::PoleParams p{};
  p.H = c->H.as<double2>();
  p.P = c->P.as<double2>();
  p.Sinf = c->Sinf_p.as<double2>();
  p.poles = c->poles.as<double>();
  p.Vp = c->Vp.as<double2>();
  p.kinfo = c->kinfo_d.as<KInfo>();
  p.sinfo = c->sinfo_d.as<SInfo>();
  p.pinfo = c->pinfo_d.as<gf::PInfo>();
  p.mu = c->mu.as<double>();
  p.n_k = c->n_k;
  p.n_iw = c->n_iw;
  p.mode = mode;
  p.max_sweeps = 40;
  p.kN = c->kN.as<double>();
  p.kdN = c->kdN.as<double>();
  p.kNc = c->kNc.as<double>();
  if (mode & gf::kRho) {
    GF_CU(ensure(c->rho_out, sizeof(double2) * c->totH));
    p.rho = c->rho_out.as<double2>();
  }
  p.eout = c->eout.as<double>();
  p.phiout = c->phiout.as<double2>();
  p.eoff = c->eoff_d.as<int64_t>();
  p.phioff = c->phioff_d.as<int64_t>();
  p.gloc = c->gacc.as<double2>();
  p.wbout = c->wbout.as<double>();
  p.kHks = c->kHks.as<double>();
  p.kEps = c->kEps.as<double>();
  p.warm = warm;
  p.save_v = save_v;
  if (warm || save_v) {
    p.vstore = c->pole_vs.as<double2>();
    p.estore = c->pole_es.as<double>();
    p.voff = c->voff_d.as<int64_t>();
    p.mu_prev = c->mu_prev.as<double>();
  }
  p.status = c->status.as<int>();
  const size_t smem = gf::heev_smem(c->nps_max);
  const size_t limit = (size_t)c->smem_optin - 16384;  // static shared arrays of the kernel
  p.in_smem = smem <= limit ? 1 : 0;
  int grid = std::min(c->n_k, c->sm_count * (p.in_smem ? std::max(1, (int)(limit / smem)) : 2));
  grid = std::max(grid, 1);
  if (!p.in_smem) {
    p.ws_stride = (int64_t)gf::heev_ws_elems(c->nps_max);
    GF_CU(ensure(c->pole_ws, sizeof(double2) * (size_t)grid * p.ws_stride));
    p.ws = c->pole_ws.as<double2>();
  }
  reserve_events(c, c->ev_used + 2);
  while ((int)c->ev.size() < c->ev_used + 2) {
    cudaEvent_t e;
    GF_CU(cudaEventCreate(&e));
    c->ev.push_back(e);
  }
  GF_CU(cudaEventRecord(c->ev[c->ev_used], c->stream));
  GF_CU(gf::launch_pole_eig(p, grid, p.in_smem ? smem : 0, c->stream));
  c->last_launches += 1;
  if ((mode & gf::kGloc) && gloc_kernel) {
    const int ns = gf::pole_gloc_splits(c->n_sys, c->n_iw, c->sm_count, c->mmax);
    GF_CU(ensure(c->pole_part, sizeof(double2) * (size_t)ns * c->totSig));
    GF_CU(gf::launch_pole_gloc(p, c->n_sys, c->mmax, ns, c->pole_part.as<double2>(), c->totSig,
                               c->stream));
    c->last_launches += 2;
  }
  GF_CU(cudaEventRecord(c->ev[c->ev_used + 1], c->stream));
  c->ev_used += 2;
  c->last_points += (int64_t)c->n_k;
  return GF_OK;
}

gf_status pole_check(gf_ctx* c) {
  gf_status st = sync_and_check(c);
  if (st) return st;
  int flags = 0;
  std::memcpy(&flags, c->hp_status(), sizeof(int));
  if (flags & 2) return fail(c, GF_ENOTCONV, "Jacobi eigensolver did not converge in 40 sweeps");
  return GF_OK;
}

gf_status pole_occupation_impl(gf_ctx* c, const double* mu, double* n_out, double* dn_out,
                               int warm = 0, int save_v = 0) {
  gf_status st = upload_mu(c, mu);
  if (st) return st;
  st = pole_run(c, gf::kOcc, true, warm, save_v);
  if (st) return st;
  GF_CU(gf::launch_sys_reduce(c->kinfo_d.as<KInfo>(), c->sinfo_d.as<SInfo>(), c->n_sys,
                              c->kN.as<double>(), c->kdN.as<double>(), c->sysout.as<double>(),
                              c->stream));
  c->last_launches += 1;
  GF_CU(cudaMemcpyAsync(c->hp_sys(), c->sysout.p, sizeof(double) * 2 * c->n_sys,
                        cudaMemcpyDeviceToHost, c->stream));
  st = pole_check(c);
  if (st) return st;
  for (int s = 0; s < c->n_sys; ++s) {
    if (n_out) n_out[s] = c->hp_sys()[2 * s];
    if (dn_out) dn_out[s] = c->hp_sys()[2 * s + 1];
  }
  return GF_OK;
}

}  // namespace

extern "C" {

gf_status gf_set_sigma_poles(gf_ctx* c, const int32_t* n_poles, const double* poles,
                             const void* v, const void* sinf) try {
  NvtxRange nvtx_range_("gf_set_sigma_poles");
  if (!c) return GF_EINVAL;
  if (!n_poles || !sinf) return fail(c, GF_EINVAL, "n_poles or sigma_inf_ptr is NULL");
  DeviceGuard guard(c->device);
  std::vector<gf::PInfo> pinfo(c->n_sys);
  int64_t offp = 0, offV = 0;
  for (int s = 0; s < c->n_sys; ++s) {
    if (n_poles[s] < 0) return fail(c, GF_EINVAL, "n_poles must be >= 0");
    if (c->sinfo[s].m > 32) return fail(c, GF_EINVAL, "the pole path takes m <= 32 orbitals");
    pinfo[s].np = n_poles[s];
    pinfo[s].pad = 0;
    pinfo[s].offp = offp;
    pinfo[s].offV = offV;
    offp += n_poles[s];
    offV += (int64_t)n_poles[s] * c->sinfo[s].m;
  }
  if (offp > 0 && (!poles || !v)) return fail(c, GF_EINVAL, "poles_ptr or v_ptr is NULL");
  std::vector<int64_t> eoff(c->n_k), phioff(c->n_k), voff(c->n_k);
  int64_t te = 0, tphi = 0, tv = 0;
  int nps = 1;
  for (int k = 0; k < c->n_k; ++k) {
    const int s = c->ksys[k];
    const int n = c->nb[k] + pinfo[s].np;
    if (n > gf::heev_max_n())
      return fail(c, GF_EINVAL, "N_b + n_poles exceeds 256, the eigensolver's largest matrix");
    nps = std::max(nps, n);
    eoff[k] = te;
    phioff[k] = tphi;
    voff[k] = tv;
    te += n;
    tphi += (int64_t)c->sinfo[s].m * n;
    tv += (int64_t)n * n;
  }
  std::vector<double> hp(std::max<int64_t>(offp, 1));
  if (offp > 0) {
    GF_CU(cudaMemcpy(hp.data(), poles, sizeof(double) * offp, cudaMemcpyDefault));
    for (int64_t i = 0; i < offp; ++i)
      if (!std::isfinite(hp[i])) return fail(c, GF_EINVAL, "a pole energy is not finite");
  }
  GF_CU(ensure(c->poles, sizeof(double) * std::max<int64_t>(offp, 1)));
  GF_CU(ensure(c->Vp, sizeof(double2) * std::max<int64_t>(offV, 1)));
  GF_CU(ensure(c->Sinf_p, sizeof(double2) * c->totSinf));
  GF_CU(ensure(c->pinfo_d, sizeof(gf::PInfo) * c->n_sys));
  GF_CU(ensure(c->eoff_d, sizeof(int64_t) * c->n_k));
  GF_CU(ensure(c->phioff_d, sizeof(int64_t) * c->n_k));
  GF_CU(ensure(c->eout, sizeof(double) * te));
  GF_CU(ensure(c->wbout, sizeof(double) * te));
  GF_CU(ensure(c->kHks, sizeof(double) * c->n_k));
  GF_CU(ensure(c->kEps, sizeof(double) * c->n_k));
  GF_CU(ensure(c->phiout, sizeof(double2) * tphi));
  GF_CU(ensure(c->kN, sizeof(double) * c->n_k));
  GF_CU(ensure(c->kdN, sizeof(double) * c->n_k));
  GF_CU(ensure(c->kNc, sizeof(double) * c->n_k));
  GF_CU(ensure(c->gacc, sizeof(double2) * c->totSig));
  if (offp > 0) {
    GF_CU(cudaMemcpyAsync(c->poles.p, hp.data(), sizeof(double) * offp, cudaMemcpyHostToDevice,
                          c->stream));
    std::vector<int64_t> sysV(c->n_sys + 1);
    for (int s = 0; s < c->n_sys; ++s) sysV[s] = pinfo[s].offV;
    sysV[c->n_sys] = offV;
    gf_status st = load_complex(c, v, sysV, c->Vp.as<double2>());
    if (st) return st;
  }
  gf_status st = load_complex(c, sinf, c->sysSinf, c->Sinf_p.as<double2>());
  if (st) return st;
  GF_CU(cudaMemcpyAsync(c->pinfo_d.p, pinfo.data(), sizeof(gf::PInfo) * c->n_sys,
                        cudaMemcpyHostToDevice, c->stream));
  GF_CU(cudaMemcpyAsync(c->eoff_d.p, eoff.data(), sizeof(int64_t) * c->n_k, cudaMemcpyHostToDevice,
                        c->stream));
  GF_CU(cudaMemcpyAsync(c->phioff_d.p, phioff.data(), sizeof(int64_t) * c->n_k,
                        cudaMemcpyHostToDevice, c->stream));
  GF_CU(ensure(c->voff_d, sizeof(int64_t) * c->n_k));
  GF_CU(cudaMemcpyAsync(c->voff_d.p, voff.data(), sizeof(int64_t) * c->n_k, cudaMemcpyHostToDevice,
                        c->stream));
  c->pole_v_elems = tv;
  c->pole_e_elems = te;
  GF_CU(cudaStreamSynchronize(c->stream));
  c->pinfo = pinfo;
  c->nps_max = nps;
  c->have_poles = true;
  return GF_OK;
} catch (...) {
  return caught(c);
}

gf_status gf_pole_occupation(gf_ctx* c, const double* mu, double* n_out, double* dn_out) try {
  NvtxRange nvtx_range_("gf_pole_occupation");
  if (!c) return GF_EINVAL;
  if (!n_out) return fail(c, GF_EINVAL, "n_out is NULL");
  DeviceGuard guard(c->device);
  reset_stats(c);
  return pole_occupation_impl(c, mu, n_out, dn_out);
} catch (...) {
  return caught(c);
}

gf_status gf_pole_find_mu(gf_ctx* c, const double* n_target, double tol, int32_t max_iter,
                          double* mu_inout, int32_t* iters_out) try {
  NvtxRange nvtx_range_("gf_pole_find_mu");
  if (!c) return GF_EINVAL;
  DeviceGuard guard(c->device);
  reset_stats(c);
  // every evaluation after the first starts Jacobi from the previous eigenpairs
  GF_CU(ensure(c->pole_vs, sizeof(double2) * std::max<int64_t>(c->pole_v_elems, 1)));
  GF_CU(ensure(c->pole_es, sizeof(double) * std::max<int64_t>(c->pole_e_elems, 1)));
  GF_CU(ensure(c->mu_prev, sizeof(double) * c->n_sys));
  int evals = 0;
  return newton_mu(c, n_target, tol, max_iter, mu_inout, iters_out,
                   [c, &evals](const double* mu, double* n, double* dn) {
                     const int warm = evals > 0 ? 1 : 0;
                     gf_status st2 = pole_occupation_impl(c, mu, n, dn, warm, 1);
                     if (st2) return st2;
                     ++evals;
                     // the stored eigenpairs now belong to this mu
                     cudaError_t e = cudaMemcpy(c->mu_prev.p, mu, sizeof(double) * c->n_sys,
                                                cudaMemcpyHostToDevice);
                     if (e != cudaSuccess) return fail(c, GF_ECUDA, cudaGetErrorString(e));
                     return GF_OK;
                   });
} catch (...) {
  return caught(c);
}

gf_status gf_pole_density_matrix(gf_ctx* c, const double* mu, void* rho_out, double* n_corr_out) try {
  NvtxRange nvtx_range_("gf_pole_density_matrix");
  if (!c) return GF_EINVAL;
  DeviceGuard guard(c->device);
  reset_stats(c);
  gf_status st = upload_mu(c, mu);
  if (st) return st;
  st = pole_run(c, gf::kRho);
  if (st) return st;
  GF_CU(gf::launch_sys_reduce(c->kinfo_d.as<KInfo>(), c->sinfo_d.as<SInfo>(), c->n_sys,
                              c->kNc.as<double>(), nullptr, c->sysout.as<double>(), c->stream));
  c->last_launches += 1;
  if (rho_out)
    GF_CU(cudaMemcpyAsync(rho_out, c->rho_out.p, sizeof(double2) * c->totH, cudaMemcpyDefault,
                          c->stream));
  GF_CU(cudaMemcpyAsync(c->hp_sys(), c->sysout.p, sizeof(double) * 2 * c->n_sys,
                        cudaMemcpyDeviceToHost, c->stream));
  st = pole_check(c);
  if (st) return st;
  if (n_corr_out)
    for (int s = 0; s < c->n_sys; ++s) n_corr_out[s] = c->hp_sys()[2 * s];
  return GF_OK;
} catch (...) {
  return caught(c);
}

gf_status gf_pole_local(gf_ctx* c, const double* mu, void* gloc_out) try {
  NvtxRange nvtx_range_("gf_pole_local");
  if (!c) return GF_EINVAL;
  if (!gloc_out) return fail(c, GF_EINVAL, "gloc_out_ptr is NULL");
  DeviceGuard guard(c->device);
  reset_stats(c);
  gf_status st = upload_mu(c, mu);
  if (st) return st;
  st = pole_run(c, gf::kGloc);
  if (st) return st;
  GF_CU(cudaMemcpyAsync(gloc_out, c->gacc.p, sizeof(double2) * c->totSig, cudaMemcpyDefault,
                        c->stream));
  return pole_check(c);
} catch (...) {
  return caught(c);
}

gf_status gf_set_projectors_lowdin(gf_ctx* c, const void* w, void* p_out) try {
  NvtxRange nvtx_range_("gf_set_projectors_lowdin");
  if (!c) return GF_EINVAL;
  if (!w) return fail(c, GF_EINVAL, "w_ptr is NULL");
  if (c->mmax > 32) return fail(c, GF_EINVAL, "the projector orthonormalisation takes m <= 32");
  DeviceGuard guard(c->device);
  GF_CU(ensure(c->wraw, sizeof(double2) * c->totP));
  gf_status st = load_complex(c, w, c->sysP, c->wraw.as<double2>());
  if (st) return st;
  GF_CU(cudaMemsetAsync(c->status.p, 0, sizeof(int), c->stream));
  GF_CU(gf::launch_lowdin(c->kinfo_d.as<KInfo>(), c->sinfo_d.as<SInfo>(), c->n_k, c->mmax,
                          c->wraw.as<double2>(), c->P.as<double2>(), c->status.as<int>(), c->stream));
  st = derive_f32(c, c->P, c->Pd, &c->Ps, c->totP);
  if (st) return st;
  if (p_out)
    GF_CU(cudaMemcpyAsync(p_out, c->P.p, sizeof(double2) * c->totP, cudaMemcpyDefault, c->stream));
  st = sync_and_check(c);
  if (st == GF_ESINGULAR)
    return fail(c, GF_ESINGULAR, "the projections of a k-point are linearly dependent (overlap "
                                 "eigenvalue <= 1e-12 of the largest)");
  if (st) return st;
  c->have_P = true;
  c->lr_dirty = true;
  c->einf_dirty = true;
  return GF_OK;
} catch (...) {
  return caught(c);
}

gf_status gf_impurity_levels(gf_ctx* c, const double* v_dc, void* e_imp_out) try {
  NvtxRange nvtx_range_("gf_impurity_levels");
  if (!c) return GF_EINVAL;
  if (!e_imp_out) return fail(c, GF_EINVAL, "e_imp_out_ptr is NULL");
  if (!c->have_H || !c->have_P)
    return fail(c, GF_ESTATE, "gf_set_hamiltonian and gf_set_projectors must be called first");
  DeviceGuard guard(c->device);
  GF_CU(ensure(c->eimp, sizeof(double2) * c->totSinf));
  GF_CU(ensure(c->eimp_part, sizeof(double2) * (size_t)c->n_k * c->mmax * c->mmax));
  GF_CU(ensure(c->vdc, sizeof(double) * c->n_sys));
  if (v_dc) {
    for (int s = 0; s < c->n_sys; ++s) {
      if (!std::isfinite(v_dc[s])) return fail(c, GF_EINVAL, "v_dc is not finite");
      c->hp_nbar()[s] = v_dc[s];
    }
    GF_CU(cudaMemcpyAsync(c->vdc.p, c->hp_nbar(), sizeof(double) * c->n_sys, cudaMemcpyHostToDevice,
                          c->stream));
  }
  GF_CU(gf::launch_eimp(c->kinfo_d.as<KInfo>(), c->sinfo_d.as<SInfo>(), c->n_k, c->n_sys,
                        c->H.as<double2>(), c->P.as<double2>(), c->nbmax, c->mmax,
                        c->eimp_part.as<double2>(), v_dc ? c->vdc.as<double>() : nullptr,
                        c->eimp.as<double2>(), c->stream));
  if (e_imp_out != c->eimp.p)
    GF_CU(cudaMemcpyAsync(e_imp_out, c->eimp.p, sizeof(double2) * c->totSinf, cudaMemcpyDefault,
                          c->stream));
  return sync_and_check(c);
} catch (...) {
  return caught(c);
}

gf_status gf_hybridization(gf_ctx* c, const double* mu, const void* gloc, const double* v_dc,
                           void* delta_out) try {
  NvtxRange nvtx_range_("gf_hybridization");
  if (!c) return GF_EINVAL;
  if (!gloc || !delta_out) return fail(c, GF_EINVAL, "gloc_ptr or delta_out_ptr is NULL");
  if (c->mmax > 32) return fail(c, GF_EINVAL, "the hybridization step takes m <= 32");
  if (!c->have_S) return fail(c, GF_ESTATE, "gf_set_sigma must be called first");
  DeviceGuard guard(c->device);
  GF_CU(ensure(c->eimp, sizeof(double2) * c->totSinf));
  gf_status st = gf_impurity_levels(c, v_dc, c->eimp.p);
  if (st) return st;
  st = upload_mu(c, mu);
  if (st) return st;
  GF_CU(ensure(c->gl_in, sizeof(double2) * c->totSig));
  GF_CU(ensure(c->delta, sizeof(double2) * c->totSig));
  GF_CU(cudaMemcpyAsync(c->gl_in.p, gloc, sizeof(double2) * c->totSig, cudaMemcpyDefault, c->stream));
  GF_CU(cudaMemsetAsync(c->status.p, 0, sizeof(int), c->stream));
  GF_CU(gf::launch_hybridization(c->sinfo_d.as<SInfo>(), c->n_sys, c->n_iw, c->mmax,
                                 c->mu.as<double>(), c->eimp.as<double2>(), c->Sig.as<double2>(),
                                 c->gl_in.as<double2>(), c->delta.as<double2>(), c->status.as<int>(),
                                 c->stream));
  GF_CU(cudaMemcpyAsync(delta_out, c->delta.p, sizeof(double2) * c->totSig, cudaMemcpyDefault,
                        c->stream));
  st = sync_and_check(c);
  if (st == GF_ESINGULAR) return fail(c, GF_ESINGULAR, "G_loc(i w_n) is singular at some frequency");
  return st;
} catch (...) {
  return caught(c);
}

gf_status gf_double_counting(double U, double J, int32_t l, double n, double* u_bar, double* v_dc,
                             double* e_dc) {
  if (!(std::isfinite(U) && std::isfinite(J) && std::isfinite(n)) || l < 0) {
    gf::set_global_error("gf_double_counting: U, J, n must be finite and l >= 0");
    return GF_EINVAL;
  }
  const double M = 2.0 * l + 1.0;
  const double ub = (U + 2.0 * (M - 1.0) * (U - 2.0 * J) - (M - 1.0) * J) / (2.0 * M - 1.0);
  if (u_bar) *u_bar = ub;
  if (v_dc) *v_dc = ub * (n - 0.5);
  if (e_dc) *e_dc = 0.5 * ub * n * (n - 1.0);
  return GF_OK;
}

gf_status gf_pole_spectral(gf_ctx* c, const double* mu, int32_t n_eps, const double* eps,
                           double eta, double* dos_out, double* pdos_out) try {
  NvtxRange nvtx_range_("gf_pole_spectral");
  if (!c) return GF_EINVAL;
  if (n_eps < 1 || !eps || !dos_out) return fail(c, GF_EINVAL, "n_eps >= 1, eps and dos_out required");
  if (!(eta > 0.0) || !std::isfinite(eta)) return fail(c, GF_EINVAL, "eta must be > 0");
  DeviceGuard guard(c->device);
  reset_stats(c);
  gf_status st = upload_mu(c, mu);
  if (st) return st;
  st = pole_run(c, gf::kGloc, false);
  if (st) return st;
  int64_t tot_m = 0;
  std::vector<int64_t> off(c->n_sys);
  for (int s2 = 0; s2 < c->n_sys; ++s2) {
    off[s2] = tot_m * n_eps;
    tot_m += c->sinfo[s2].m;
  }
  GF_CU(ensure(c->eps_grid, sizeof(double) * n_eps));
  GF_CU(ensure(c->dos, sizeof(double) * (size_t)n_eps * c->n_sys));
  GF_CU(ensure(c->pdos, sizeof(double) * (size_t)n_eps * tot_m));
  GF_CU(ensure(c->pdos_off, sizeof(int64_t) * c->n_sys));
  GF_CU(cudaMemcpyAsync(c->eps_grid.p, eps, sizeof(double) * n_eps, cudaMemcpyDefault, c->stream));
  GF_CU(cudaMemcpyAsync(c->pdos_off.p, off.data(), sizeof(int64_t) * c->n_sys, cudaMemcpyHostToDevice,
                        c->stream));
  gf::PoleParams p{};
  p.kinfo = c->kinfo_d.as<KInfo>();
  p.sinfo = c->sinfo_d.as<SInfo>();
  p.pinfo = c->pinfo_d.as<gf::PInfo>();
  p.mu = c->mu.as<double>();
  p.eout = c->eout.as<double>();
  p.wbout = c->wbout.as<double>();
  p.phiout = c->phiout.as<double2>();
  p.eoff = c->eoff_d.as<int64_t>();
  p.phioff = c->phioff_d.as<int64_t>();
  GF_CU(gf::launch_pole_dos(p, c->n_sys, c->eps_grid.as<double>(), n_eps, eta,
                            c->pdos_off.as<int64_t>(), c->dos.as<double>(),
                            pdos_out ? c->pdos.as<double>() : nullptr, c->stream));
  c->last_launches += 1;
  GF_CU(cudaMemcpyAsync(dos_out, c->dos.p, sizeof(double) * (size_t)n_eps * c->n_sys,
                        cudaMemcpyDefault, c->stream));
  if (pdos_out)
    GF_CU(cudaMemcpyAsync(pdos_out, c->pdos.p, sizeof(double) * (size_t)n_eps * tot_m,
                          cudaMemcpyDefault, c->stream));
  return pole_check(c);
} catch (...) {
  return caught(c);
}

gf_status gf_pole_energy(gf_ctx* c, const double* mu, double* h_ks_out, double* e_ps_out) try {
  NvtxRange nvtx_range_("gf_pole_energy");
  if (!c) return GF_EINVAL;
  if (!h_ks_out && !e_ps_out) return fail(c, GF_EINVAL, "h_ks_out and e_ps_out are both NULL");
  DeviceGuard guard(c->device);
  reset_stats(c);
  gf_status st = upload_mu(c, mu);
  if (st) return st;
  GF_CU(ensure(c->rho_out, sizeof(double2) * c->totH));
  st = pole_run(c, gf::kRho);
  if (st) return st;
  GF_CU(gf::launch_sys_reduce(c->kinfo_d.as<KInfo>(), c->sinfo_d.as<SInfo>(), c->n_sys,
                              c->kHks.as<double>(), c->kEps.as<double>(), c->sysout.as<double>(),
                              c->stream));
  c->last_launches += 1;
  GF_CU(cudaMemcpyAsync(c->hp_sys(), c->sysout.p, sizeof(double) * 2 * c->n_sys,
                        cudaMemcpyDeviceToHost, c->stream));
  st = pole_check(c);
  if (st) return st;
  for (int s2 = 0; s2 < c->n_sys; ++s2) {
    if (h_ks_out) h_ks_out[s2] = c->hp_sys()[2 * s2];
    if (e_ps_out) e_ps_out[s2] = c->hp_sys()[2 * s2 + 1];
  }
  return GF_OK;
} catch (...) {
  return caught(c);
}

gf_status gf_heev_batched(const void* a_dev, int32_t n_mat, int32_t n, int32_t max_sweeps,
                          double* w_dev, void* v_dev, void* stream) try {
  NvtxRange nvtx_range_("gf_heev_batched");
  if (n_mat < 0 || n < 1 || n > gf::heev_max_n() || max_sweeps < 1 ||
      (n_mat > 0 && (!a_dev || !w_dev || !v_dev))) {
    gf::set_global_error("gf_heev_batched: invalid arguments (1 <= n <= 256, max_sweeps >= 1, "
                         "non-null device pointers)");
    return GF_EINVAL;
  }
  if (n_mat == 0) return GF_OK;
  const void* ptrs[3] = {a_dev, w_dev, v_dev};
  for (const void* q : ptrs) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, q) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
      cudaGetLastError();
      gf::set_global_error("gf_heev_batched: a, w and v must be device pointers");
      return GF_EINVAL;
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 1, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t smem = gf::heev_smem(n);
  const int in_smem = smem + 8192 <= (size_t)optin ? 1 : 0;
  const int grid = std::max(1, std::min(n_mat, sms * (in_smem ? std::max(1, (int)((optin - 8192) / smem)) : 2)));
  void* mem = nullptr;
  const size_t ws = in_smem ? 0 : sizeof(double2) * gf::heev_ws_elems(n) * grid;
  cudaError_t e = cudaMallocAsync(&mem, 16 + ws, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(mem, 0, sizeof(int), s);
  int* status = static_cast<int*>(mem);
  double2* gws = reinterpret_cast<double2*>(static_cast<char*>(mem) + 16);
  if (e == cudaSuccess)
    e = gf::launch_heev_batched(static_cast<const double2*>(a_dev), n_mat, n, max_sweeps, w_dev,
                                static_cast<double2*>(v_dev), gws, grid, in_smem, status, s);
  int flags = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flags, status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (mem) cudaFreeAsync(mem, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    gf::set_global_error((std::string("gf_heev_batched: ") + cudaGetErrorString(e)).c_str());
    return e == cudaErrorMemoryAllocation ? GF_ENOMEM : GF_ECUDA;
  }
  if (flags & 2) {
    gf::set_global_error("gf_heev_batched: Jacobi did not converge within max_sweeps");
    return GF_ENOTCONV;
  }
  return GF_OK;
} catch (...) {
  return caught(nullptr);
}

}  // extern "C"
