// C-ABI of libgf (declared in include/gf.h): context, argument validation,
// host<->device marshalling, work-item scheduling and the mu search.
#include "gf_ctx.cuh"

namespace {

thread_local std::string g_create_error;

double trigamma(double x) {
  double acc = 0.0;
  while (x < 20.0) {
    acc += 1.0 / (x * x);
    x += 1.0;
  }
  const double ix = 1.0 / x, ix2 = ix * ix;
  const double series =
      ix + 0.5 * ix2 +
      ix * ix2 * (1.0 / 6 - ix2 * (1.0 / 30 - ix2 * (1.0 / 42 - ix2 * (1.0 / 30 - ix2 * 5.0 / 66))));
  return acc + series;
}

}  // namespace

namespace gf {

// (2/beta) sum_{n<N} 1/w_n^2 - beta/4 = -(2/beta)(beta/pi)^2 sum_{n>=N} (2n+1)^-2
//                                     = -(beta/(2 pi^2)) psi'(N + 1/2)
double tail_coefficient(double beta, int n_iw, int tail_order) {
  if (tail_order != 2) return 0.0;
  return -beta / (2.0 * M_PI * M_PI) * trigamma(n_iw + 0.5);
}

void set_global_error(const char* msg) noexcept {
  try {
    g_create_error = msg ? msg : "";
  } catch (...) {
    g_create_error.clear();
  }
}

}  // namespace gf

namespace {

gf_status ensure_einf(gf_ctx* c) {
  if (!c->einf_dirty) return GF_OK;
  GF_CU(gf::launch_einf(c->kinfo_d.as<KInfo>(), c->sinfo_d.as<SInfo>(), c->H.as<double2>(),
                        c->P.as<double2>(), c->Sinf.as<double2>(), c->n_k, c->Einf.as<double2>(),
                        c->trHE.as<double>(), c->stream));
  c->last_launches += 1;
  c->einf_dirty = false;
  return GF_OK;
}

// Low-rank path: eigen-decomposition of every H_k and Pt = P_k U, once per
// Hamiltonian / projector upload.
gf_status ensure_lr(gf_ctx* c) {
  if (!c->lowrank || !c->lr_dirty) return GF_OK;
  if (c->nbmax > gf::heev_max_n())
    return fail(c, GF_EINVAL, "GF_FLAG_LOWRANK takes N_b <= 256");
  GF_CU(ensure(c->lr_eps, sizeof(double) * c->totNb));
  GF_CU(ensure(c->lr_U, sizeof(double2) * c->totH));
  GF_CU(ensure(c->lr_Pt, sizeof(double2) * c->totP));
  const size_t smem = gf::heev_smem(c->nbmax);
  const size_t limit = (size_t)c->smem_optin - 8192;
  const int in_smem = smem <= limit ? 1 : 0;
  int grid = std::min(c->n_k, c->sm_count * (in_smem ? std::max(1, (int)(limit / smem)) : 2));
  grid = std::max(grid, 1);
  if (!in_smem) GF_CU(ensure(c->lr_ws, sizeof(double2) * gf::heev_ws_elems(c->nbmax) * grid));
  GF_CU(gf::launch_lr_setup(c->H.as<double2>(), c->P.as<double2>(), c->kinfo_d.as<KInfo>(),
                            c->sinfo_d.as<SInfo>(), c->offD_d.as<int64_t>(), c->n_k, c->nbmax,
                            c->lr_eps.as<double>(), c->lr_U.as<double2>(), c->lr_Pt.as<double2>(),
                            c->lr_ws.as<double2>(), grid, in_smem, c->status.as<int>(), c->stream));
  c->last_launches += 1;
  c->lr_dirty = false;
  return GF_OK;
}

// rho_k partial sums: the low-rank kernel leaves them in the eigenbasis of H_k;
// sum the chunks and rotate back, leaving one chunk for k_rho_finalize.
gf_status rho_partials(gf_ctx* c, int* n_chunks) {
  *n_chunks = c->n_chunks;
  if (!c->lowrank) return GF_OK;
  GF_CU(ensure(c->lr_T, sizeof(double2) * c->totH));
  GF_CU(gf::launch_lr_rotate(c->kinfo_d.as<KInfo>(), c->n_k, c->lr_U.as<double2>(),
                             c->rho_part.as<double2>(), c->totH, c->n_chunks, c->lr_T.as<double2>(),
                             c->stream));
  c->last_launches += 1;
  *n_chunks = 1;
  return GF_OK;
}

gf_status check_ready(gf_ctx* c) {
  if (!c->have_H || !c->have_P || !c->have_S)
    return fail(c, GF_ESTATE, "gf_set_hamiltonian, gf_set_projectors and gf_set_sigma must all be "
                              "called before a compute call");
  return GF_OK;
}

// Kernel configuration of one launch, i.e. of one bucket of band-window sizes.
struct LaunchCfg {
  int kind = 0;        // 0 FP64, 1 FP32-pair shared-memory, 2 FP32-pair register-resident,
                       // 3 low-rank, 4 FP32 register-resident with refined projections,
                       // 5 tensor-core (tcgen05) blocked elimination, N(mu) passes,
                       // 6 one warp per matrix (windows <= 40), 7 two or three warps per
                       // matrix (windows 41-96): N(mu) passes; 8 one warp per matrix and
                       // the CTA's refined projections: fused passes, windows <= 40
  int shape = -1;      // register tile shape (kinds 2 and 4); matrices per CTA (kind 5)
  int threads = gf::kThreads;
  size_t smem = 0;
  int grid = 1;
  int a_in_smem = 1;
  int nbmax = 1;
  int pair_table = 0;  // low-rank kernel: pair table of the item in shared memory
};

gf_status launch_cfg(gf_ctx* c, const LaunchCfg& cfg, gf::PointParams p, int n_items) {
  p.nbmax = cfg.nbmax;
  p.a_in_smem = cfg.a_in_smem;
  p.nmat = 1;
  if (!cfg.a_in_smem) {
    p.a_stride = (int64_t)cfg.nbmax * (cfg.nbmax | 1);
    GF_CU(ensure(c->a_scratch, (size_t)cfg.grid * p.a_stride * sizeof(double2)));
    p.a_scratch = c->a_scratch.as<double2>();
  }
  p.n_items = n_items;
  const int grid = std::min(cfg.grid, std::max(1, n_items));
  if (cfg.kind == 3) {
    gf::LowRank lr{c->lr_eps.as<double>(), c->offD_d.as<int64_t>(), c->lr_Pt.as<double2>(),
                   cfg.pair_table, c->precision != GF_PREC_FP64 ? 1 : 0};
    GF_CU(gf::launch_point_lr(p, lr, grid, cfg.smem, c->stream));
    return GF_OK;
  }
  if (cfg.kind == 8) {
    GF_CU(gf::launch_point_f32w(cfg.nbmax, p, grid, cfg.smem, c->stream));
  } else if (cfg.kind == 7) {
    GF_CU(gf::launch_point_wm(cfg.nbmax, p, grid, cfg.smem, c->stream));
  } else if (cfg.kind == 6) {
    GF_CU(gf::launch_point_w32(cfg.nbmax, p, grid, cfg.smem, c->stream));
  } else if (cfg.kind == 5) {
    // GF_TC_TEST_SKIP_MMA=1 (failure-detection tests): the kernel's bounded waits run out
    const char* skip = std::getenv("GF_TC_TEST_SKIP_MMA");
    p.tc_skip_mma = (skip && std::atoi(skip) == 1) ? 1 : 0;
    GF_CU(gf::launch_point_tc(cfg.shape, p, grid, cfg.smem, c->stream));
  } else if (cfg.kind == 4) GF_CU(gf::launch_point_f32r(cfg.shape, p, grid, cfg.threads, cfg.smem, c->stream));
  else if (cfg.kind == 2) GF_CU(gf::launch_point_df64r(cfg.shape, p, grid, cfg.threads, cfg.smem, c->stream));
  else if (cfg.kind == 1) GF_CU(gf::launch_point_df64(p, grid, cfg.smem, c->stream));
  else GF_CU(gf::launch_point_fp64(p, grid, cfg.smem, c->stream));
  return GF_OK;
}

std::string cfg_name(const LaunchCfg& g) {
  char buf[96];
  if (g.kind == 8)
    std::snprintf(buf, sizeof(buf), "FP32 one warp per matrix + CTA projections, %d threads, %d CTAs", g.threads,
                  g.grid);
  else if (g.kind == 6)
    std::snprintf(buf, sizeof(buf), "FP32 one warp per matrix, %d threads, %d CTAs", g.threads, g.grid);
  else if (g.kind == 7)
    std::snprintf(buf, sizeof(buf), "FP32 %d warps per matrix, %d CTAs", g.threads / 32, g.grid);
  else if (g.kind == 5)
    std::snprintf(buf, sizeof(buf), "tensor cores (TF32 split), %d matrices x 128 threads, %d CTAs", g.shape,
                  g.grid);
  else if (g.kind == 4)
    std::snprintf(buf, sizeof(buf), "FP32 register %dx%d tiles x %d threads, %d CTAs",
                  gf::f32r_tile(g.shape, 0), gf::f32r_tile(g.shape, 1), g.threads, g.grid);
  else if (g.kind == 2)
    std::snprintf(buf, sizeof(buf), "register %dx%d tiles x %d threads", gf::df64r_tile(g.shape, 0),
                  gf::df64r_tile(g.shape, 1), g.threads);
  else
    std::snprintf(buf, sizeof(buf), "%s, matrix in %s, %d CTAs", g.kind ? "FP32-pair" : "FP64",
                  g.a_in_smem ? "shared memory" : "L2 (global scratch)", g.grid);
  return buf;
}

// Autotuner: the first time a (mode, window bucket) runs with more than one
// candidate configuration, the first items of that bucket are run with each
// candidate, timed with CUDA events, and the fastest is kept for the context.
// The sample runs write only scratch that the real run overwrites.
// GF_AUTOTUNE=0 skips the timing and takes the last candidate.
gf_status autotune(gf_ctx* c, int key, const std::vector<LaunchCfg>& cands, gf::PointParams p,
                   const Item* items, int n_items, LaunchCfg* out) {
  auto it = c->tuned.find(key);
  if (it != c->tuned.end()) {
    *out = cands[std::min<size_t>(it->second, cands.size() - 1)];
    return GF_OK;
  }
  const char* env = std::getenv("GF_AUTOTUNE");
  if (cands.size() == 1 || (env && std::atoi(env) == 0)) {
    c->tuned[key] = (int)cands.size() - 1;
    *out = cands.back();
    c->tune_log += "mode " + std::to_string(key >> 3) + ", windows <= " + std::to_string(cands[0].nbmax) + ": " +
                   cfg_name(cands.back()) + (cands.size() == 1 ? " (only candidate); " : " (not timed); ");
    return GF_OK;
  }
  // the sample: whole waves of every candidate's grid, at least one item per CTA of the
  // largest grid (so a candidate with fewer CTAs is not charged a partial last wave), and
  // the time per item compared; a second run of a candidate only when its first took under
  // 50 ms (the first run of a kernel also loads its module, which is noise against a long
  // sample)
  int maxgrid = 1;
  for (const LaunchCfg& g : cands) maxgrid = std::max(maxgrid, g.grid);
  p.items = items;
  std::vector<float> ms(cands.size(), 0.f);
  std::vector<int> n_sample(cands.size(), 1);
  ScopedEvents ev;
  GF_CU(ev.create());
  for (size_t cand = 0; cand < cands.size(); ++cand) {
    const int g = std::max(1, std::min(cands[cand].grid, n_items));
    n_sample[cand] = std::min(n_items, g * ((maxgrid + g - 1) / g));
    for (int rep = 0; rep < 2; ++rep) {
      GF_CU(cudaMemsetAsync(c->queue.p, 0, sizeof(int), c->stream));
      GF_CU(cudaEventRecord(ev.start, c->stream));
      gf_status st = launch_cfg(c, cands[cand], p, n_sample[cand]);
      if (st) return st;
      GF_CU(cudaEventRecord(ev.stop, c->stream));
      GF_CU(cudaEventSynchronize(ev.stop));
      GF_CU(cudaEventElapsedTime(&ms[cand], ev.start, ev.stop));
      c->last_launches += 1;
      if (ms[cand] > 50.f) break;
    }
  }
  int best = 0;
  for (size_t cand = 1; cand < cands.size(); ++cand)
    if (ms[cand] / n_sample[cand] < ms[best] / n_sample[best]) best = (int)cand;
  c->tuned[key] = best;
  *out = cands[best];
  std::string line = "mode " + std::to_string(key >> 3) + ", windows <= " +
                     std::to_string(cands[0].nbmax) + ": " + cfg_name(cands[best]) + " (samples:";
  for (size_t cand = 0; cand < cands.size(); ++cand) {
    char buf[64];
    std::snprintf(buf, sizeof(buf), " %d items %.3f ms", n_sample[cand], ms[cand]);
    line += (cand ? "; " : " ") + cfg_name(cands[cand]) + buf;
  }
  c->tune_log += line + "); ";
  return GF_OK;
}

// Candidate launch configurations for the items of one window bucket (largest
// window nbmax): the point kernel of the context's precision with the matrix in
// shared memory (when it fits) and in an L2-resident global slice (more CTAs per
// SM), and with FP32 pairs the register-resident kernel (windows <= 96).  The
// mixed path takes the single-word FP32 register kernel for windows up to 128
// (falling back to the FP32-pair kernels above that).
gf_status choose_cfg(gf_ctx* c, int mode, int bucket, int nbmax, const gf::PointParams& p,
                     const Item* items, int n_items, LaunchCfg* cfg) {
  const size_t limit = (size_t)c->smem_optin - 1024;
  std::vector<LaunchCfg> cands;
  if (c->precision == GF_PREC_MIXED) {
    // GF_KERNEL restricts the mixed candidates to one kernel family: tc (tensor cores),
    // w32 (one to three warps per matrix) or f32r (register tiles)
    const char* only = std::getenv("GF_KERNEL");
    const bool use_tc = only && std::strcmp(only, "tc") == 0;
    const bool use_w32 = !only || std::strcmp(only, "w32") == 0;
    const bool use_f32r = !only || std::strcmp(only, "f32r") == 0;
    // N(mu) passes: the tensor-core elimination with 4 to 1 matrices per CTA
    for (int ng = 4; use_tc && mode == gf::kOcc && ng >= 1; --ng) {
      if (!gf::tc_fits(nbmax, ng)) continue;
      LaunchCfg t;
      t.kind = 5;
      t.shape = ng;
      t.nbmax = nbmax;
      t.threads = 128 * ng;
      t.smem = gf::point_tc_smem(nbmax, c->mmax, ng);
      if (t.smem > limit) continue;
      const int bps = gf::point_tc_blocks_per_sm(nbmax, ng, t.smem);
      if (bps < 1) continue;
      t.grid = c->sm_count * bps;
      cands.push_back(t);
    }
    // N(mu) passes of windows up to 40 bands: one warp per matrix
    if (use_w32 && mode == gf::kOcc && gf::w32_nmax(nbmax) > 0) {
      LaunchCfg w;
      w.kind = 6;
      w.nbmax = nbmax;
      w.threads = gf::w32_threads();
      w.smem = gf::point_w32_smem(nbmax, c->mmax);
      const int bps = w.smem <= limit ? gf::point_w32_blocks_per_sm(nbmax, w.smem) : 0;
      w.grid = c->sm_count * bps;
      if (bps >= 1) cands.push_back(w);
    }
    // fused passes of windows up to 40 bands: one warp per matrix, the CTA's epilogues
    if (use_w32 && mode != gf::kOcc && gf::f32w_nmax(nbmax) > 0) {
      LaunchCfg w;
      w.kind = 8;
      w.nbmax = nbmax;
      w.threads = gf::f32w_threads();
      w.smem = gf::point_f32w_smem(nbmax, c->mmax, mode);
      const int bps = w.smem <= limit ? gf::point_f32w_blocks_per_sm(nbmax, w.smem) : 0;
      w.grid = c->sm_count * bps;
      if (bps >= 1) cands.push_back(w);
    }
    // ... and of 41 to 96 bands: two or three warps per matrix, one row per lane
    if (use_w32 && mode == gf::kOcc && gf::wm_nmax(nbmax) > 0) {
      LaunchCfg w;
      w.kind = 7;
      w.nbmax = nbmax;
      w.threads = gf::wm_threads(nbmax);
      w.smem = gf::point_wm_smem(nbmax, c->mmax);
      const int bps = w.smem <= limit ? gf::point_wm_blocks_per_sm(nbmax, w.smem) : 0;
      w.grid = c->sm_count * bps;
      if (bps >= 1) cands.push_back(w);
    }
    // single-word FP32 register tiles for every shape that serves the window
    for (int sh = 0; use_f32r && sh < gf::f32r_num_shapes(); ++sh) {
      if (!gf::f32r_shape_fits(sh, nbmax)) continue;
      LaunchCfg f;
      f.kind = 4;
      f.shape = sh;
      f.nbmax = nbmax;
      f.threads = gf::f32r_threads(sh, nbmax);
      f.smem = gf::point_f32r_smem(nbmax, c->mmax, mode);
      f.a_in_smem = 1;
      if (f.smem > limit) continue;
      const int bps = gf::point_f32r_blocks_per_sm(sh, f.threads, f.smem);
      if (bps < 1) continue;
      f.grid = c->sm_count * bps;
      cands.push_back(f);
    }
    if (!cands.empty()) return autotune(c, mode * 8 + bucket, cands, p, items, n_items, cfg);
    // windows above the register tiles: the FP32-pair kernels below
  }
  const int kind = (c->precision == GF_PREC_FP64) ? 0 : 1;
  for (int in_smem = 1; in_smem >= 0; --in_smem) {
    LaunchCfg a;
    a.nbmax = nbmax;
    a.kind = kind;
    a.a_in_smem = in_smem;
    a.smem = gf::point_fp64_smem(nbmax, c->mmax, mode, in_smem);  // same layout for both kernels
    if (a.smem > limit) continue;
    const int bps = kind ? gf::point_df64_blocks_per_sm(a.smem) : gf::point_fp64_blocks_per_sm(a.smem);
    a.grid = c->sm_count * std::max(1, bps);
    // the L2 variant only when it raises occupancy
    if (!in_smem && !cands.empty() && a.grid <= cands[0].grid) continue;
    cands.push_back(a);
  }
  if (cands.empty())
    return fail(c, GF_EINVAL, "N_b or m too large for the shared-memory tiles of the point kernel");
  const int shape = kind ? gf::df64r_shape(nbmax) : -1;
  if (shape >= 0) {
    LaunchCfg b;
    b.kind = 2;
    b.shape = shape;
    b.nbmax = nbmax;
    b.threads = gf::df64r_threads(shape, nbmax);
    b.smem = gf::point_df64r_smem(nbmax, c->mmax, mode);
    b.a_in_smem = 1;
    b.grid = c->sm_count * std::max(1, gf::point_df64r_blocks_per_sm(shape, b.threads, b.smem));
    if (b.smem <= limit) cands.push_back(b);
  }
  return autotune(c, mode * 8 + bucket, cands, p, items, n_items, cfg);
}

// Algorithmic floating-point operations of one (k, i w_n) point (8 per complex
// multiply-add, 2 per complex add or real product pair).
double point_flops(int N, int M, int mode) {
  const double n = N, m = M;
  double cmac = n * n * n + m * m * n + m * n * n;  // inverse + embedding
  double f = 0.0;
  if (mode & gf::kOcc) f += 2.0 * n * n + 2.0 * n;  // Re Tr G^2, Re Tr G
  if (mode & gf::kRho) f += 2.0 * n * n;            // S += G
  if (mode & (gf::kGloc | gf::kAdj)) cmac += m * n * n + m * m * n;  // Y = G P^+, P Y
  if (mode & gf::kAdj) cmac += m * n * n + m * m * n + 2.0 * m * m * m;  // Z = P G, Z Y, A^+ Gbar A^+
  return 8.0 * cmac + f;
}

// Floating-point operations of one point of the low-rank kernel (8 per complex
// multiply-add): g0 (and g1, g2) N_b m^2 each, Sigma g0 and the elimination
// m^3 + m^2 (2m) / 2 ..., the products of the epilogue m^3 each.
double point_flops_lr(int N, int M, int mode) {
  const double n = N, m = M;
  double cmac = m * m * n + m * m * m + m * m * m;  // g0, Sigma g0, [M | Sigma] elimination
  if (mode & (gf::kOcc | gf::kAdj)) cmac += m * m * n + m * m * m;  // g1, K g1
  if (mode & gf::kOcc) cmac += m * m * n;                          // g2
  if (mode & (gf::kGloc | gf::kAdj)) cmac += 2.0 * m * m * m;       // K g0, g0 K g0
  if (mode & gf::kRho) cmac += m * m * n + m * n * n;               // K Pt, Pt^+ (K Pt)
  if (mode & gf::kAdj) cmac += 4.0 * m * m * m;                     // B, A^+ Gbar A^+
  return 8.0 * cmac;
}

// Run the point kernel over every (k, chunk) item with the given mode.  For
// kGloc / kAdj the per-(k, n) m x m results are reduced over k into c->gacc,
// k-batch by k-batch, in increasing k order.
gf_status run_points(gf_ctx* c, int mode) {
  gf_status st = check_ready(c);
  if (st) return st;
  st = ensure_einf(c);
  if (st) return st;
  GF_CU(cudaMemsetAsync(c->status.p, 0, sizeof(int), c->stream));
  st = ensure_lr(c);
  if (st) return st;
  const bool df64 = (c->precision != GF_PREC_FP64);
  gf::PointParams p{};
  p.H = c->H.as<double2>();
  p.P = c->P.as<double2>();
  p.Sig = c->Sig.as<double2>();
  if (df64) {
    p.Hd = c->Hd.as<float4>();
    p.Pd = c->Pd.as<float4>();
    p.Sd = c->Sd.as<float4>();
  }
  if (c->precision == GF_PREC_MIXED) {
    p.Hs = c->Hs.as<float2>();
    p.Ps = c->Ps.as<float2>();
    p.Ss = c->Ss.as<float2>();
  }
  p.kinfo = c->kinfo_d.as<KInfo>();
  p.sinfo = c->sinfo_d.as<SInfo>();
  p.n_chunks = c->n_chunks;
  p.queue = c->queue.as<int>();
  p.mu = c->mu.as<double>();
  p.mode = mode;
  p.mmax = c->mmax;
  p.nmat = 1;
  if (mode & gf::kOcc) {
    GF_CU(ensure(c->occ_part, sizeof(double) * 2 * (size_t)c->n_k * c->n_chunks));
    p.occ_part = c->occ_part.as<double>();
  }
  if (mode & gf::kRho) {
    p.rho_chunk_stride = c->totH;
    GF_CU(ensure(c->rho_part, sizeof(double2) * (size_t)c->totH * c->n_chunks));
    p.rho_part = c->rho_part.as<double2>();
  }
  if (mode & gf::kAdj) {
    GF_CU(ensure(c->mubar_part, sizeof(double) * (size_t)c->n_k * c->n_chunks));
    p.mubar_part = c->mubar_part.as<double>();
  }
  p.n_iw = c->n_iw;
  p.status = c->status.as<int>();
  p.gbar = nullptr;
  p.nbar = nullptr;
  if (mode & gf::kAdj) {
    p.gbar = c->have_gbar_for_call ? c->gbar.as<double2>() : nullptr;
    p.Gbd = (df64 && c->have_gbar_for_call) ? c->Gbd.as<float4>() : nullptr;
    p.nbar = c->nbar.as<double>();
  }
  const bool kred = (mode & (gf::kGloc | gf::kAdj)) != 0;
  const int nb_batches = kred ? (int)c->batch_g0.size() - 1 : 1;
  p.kperm = kred ? c->kperm_d.as<int>() : nullptr;
  // window of an item's (first) k-point: the k-points of a group share a bucket
  auto item_nb = [&](const Item& it) { return c->nb[kred ? c->kperm[it.k] : it.k]; };
  int64_t points = 0;
  for (int b = 0; b < nb_batches; ++b) {
    const int i0 = kred ? c->batch_item0[b] : c->all_item0;
    const int i1 = kred ? c->batch_item0[b + 1] : c->all_item0 + c->n_items_all;
    const int gb0 = kred ? c->batch_g0[b] : 0;
    const int gb1 = kred ? c->batch_g0[b + 1] : 0;
    if (kred) {
      GF_CU(ensure(c->gq, sizeof(double2) * (size_t)(gb1 - gb0) * c->n_iw * c->mmax * c->mmax));
      p.gq = c->gq.as<double2>();
      p.gb0 = gb0;
    }
    // items are sorted by decreasing window: one launch per window bucket, with
    // shared-memory tiles sized to the bucket's largest window
    for (int s0 = i0; s0 < i1;) {
      const int bucket = gf_bucket(item_nb(c->items[s0]));
      int s1 = s0;
      while (s1 < i1 && gf_bucket(item_nb(c->items[s1])) == bucket) ++s1;
      const Item* items_dev = c->items_d.as<Item>() + s0;
      LaunchCfg cfg;
      if (c->lowrank) {
        cfg.kind = 3;
        cfg.nbmax = c->bucket_nbmax[bucket];
        const size_t lim = (size_t)c->smem_optin - 1024;
        const int ps = c->precision != GF_PREC_FP64 ? 1 : 0;  // FP32-pair band sums
        const size_t s0 = gf::point_lr_smem(cfg.nbmax, c->mmax, mode, 0, ps);
        const size_t s1 = gf::point_lr_smem(cfg.nbmax, c->mmax, mode, 1, ps);
        if (s0 > lim)
          return fail(c, GF_EINVAL, "N_b or m too large for the shared-memory tiles of the low-rank kernel");
        const int b0 = std::max(1, gf::point_lr_blocks_per_sm(s0, ps));
        const int b1 = s1 <= lim ? gf::point_lr_blocks_per_sm(s1, ps) : 0;
        // keep the item's pair table in shared memory when that costs no occupancy
        cfg.pair_table = (b1 >= b0) ? 1 : 0;
        cfg.smem = cfg.pair_table ? s1 : s0;
        cfg.grid = c->sm_count * (cfg.pair_table ? b1 : b0);
      } else {
        st = choose_cfg(c, mode, bucket, c->bucket_nbmax[bucket], p, items_dev, s1 - s0, &cfg);
        if (st) return st;
      }
      p.items = items_dev;
      GF_CU(cudaMemsetAsync(c->queue.p, 0, sizeof(int), c->stream));
      reserve_events(c, c->ev_used + 2);
      while ((int)c->ev.size() < c->ev_used + 2) {
        cudaEvent_t e;
        GF_CU(cudaEventCreate(&e));
        c->ev.push_back(e);
      }
      // (events recorded inside a CUDA graph cannot be timed: a replay is timed as a whole)
      if (!c->capturing) GF_CU(cudaEventRecord(c->ev[c->ev_used], c->stream));
      st = launch_cfg(c, cfg, p, s1 - s0);
      if (st) return st;
      if (!c->capturing) {
        GF_CU(cudaEventRecord(c->ev[c->ev_used + 1], c->stream));
        c->ev_used += 2;
      }
      c->last_launches += 1;
      s0 = s1;
    }
    if (kred) {
      int max_total = 0;
      for (const SInfo& si : c->sinfo) max_total = std::max(max_total, c->n_iw * si.m * si.m);
      GF_CU(gf::launch_gq_reduce(c->sinfo_d.as<SInfo>(), c->n_sys, max_total, c->sysg_d.as<int>(),
                                 c->sysg_d.as<int>() + c->n_sys, c->gq.as<double2>(), gb0, gb1, c->n_iw,
                                 c->mmax, b == 0, c->gacc.as<double2>(), c->stream));
      c->last_launches += 1;
    }
    for (int i = i0; i < i1; ++i) {
      const Item& it = c->items[i];
      for (int q = 0; q < it.nk; ++q) {
        const int k = kred ? c->kperm[it.k + q] : it.k + q;
        points += it.n1 - it.n0;
        c->last_flops += (it.n1 - it.n0) * (c->lowrank ? point_flops_lr(c->nb[k], c->msys[c->ksys[k]], mode)
                                                       : point_flops(c->nb[k], c->msys[c->ksys[k]], mode));
      }
    }
  }
  c->last_points += points;
  return GF_OK;
}


// Enqueue one N(mu) evaluation (mu already in c->hp_mu): upload, point kernel,
// finalize, read-back of (N, dN/dmu) and the status word.  No synchronisation,
// so the sequence can be captured into a CUDA graph.
gf_status enqueue_occupation(gf_ctx* c) {
  GF_CU(cudaMemcpyAsync(c->mu.p, c->hp_mu(), sizeof(double) * c->n_sys, cudaMemcpyHostToDevice,
                        c->stream));
  gf_status st = run_points(c, gf::kOcc);
  if (st) return st;
  GF_CU(gf::launch_occ_finalize(c->kinfo_d.as<KInfo>(), c->sinfo_d.as<SInfo>(), c->trHE.as<double>(),
                                c->mu.as<double>(), c->occ_part.as<double>(), c->n_chunks, c->n_k,
                                c->kN.as<double>(), c->kdN.as<double>(), c->stream));
  GF_CU(gf::launch_sys_reduce(c->kinfo_d.as<KInfo>(), c->sinfo_d.as<SInfo>(), c->n_sys,
                              c->kN.as<double>(), c->kdN.as<double>(), c->sysout.as<double>(),
                              c->stream));
  c->last_launches += 2;
  GF_CU(cudaMemcpyAsync(c->hp_sys(), c->sysout.p, sizeof(double) * 2 * c->n_sys,
                        cudaMemcpyDeviceToHost, c->stream));
  GF_CU(cudaMemcpyAsync(c->hp_status(), c->status.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  return GF_OK;
}

// After the stream (or the graph's stream) drained: kernel times, status, results.
gf_status finish_occupation(gf_ctx* c, cudaStream_t s, double* n_out, double* dn_out) {
  GF_CU(cudaStreamSynchronize(s));
  for (int i = 0; i + 1 < c->ev_used; i += 2) {
    float ms = 0.f;
    GF_CU(cudaEventElapsedTime(&ms, c->ev[i], c->ev[i + 1]));
    c->last_kernel_ms += ms;
  }
  c->ev_used = 0;
  int flags = 0;
  std::memcpy(&flags, c->hp_status(), sizeof(int));
  if (flags & gf::kFlagTimeout)
    return fail(c, GF_ETIMEOUT, "a bounded wait for the tensor cores gave up in the point kernel");
  if (flags & gf::kFlagSingular)
    return fail(c, GF_ESINGULAR, "zero or non-finite pivot in a (k, i w_n) inverse");
  for (int s2 = 0; s2 < c->n_sys; ++s2) {
    if (n_out) n_out[s2] = c->hp_sys()[2 * s2];
    if (dn_out) dn_out[s2] = c->hp_sys()[2 * s2 + 1];
  }
  return GF_OK;
}

gf_status occupation_impl(gf_ctx* c, const double* mu, double* n_out, double* dn_out) {
  if (!mu) return fail(c, GF_EINVAL, "mu is NULL");
  for (int s2 = 0; s2 < c->n_sys; ++s2)
    if (!std::isfinite(mu[s2])) return fail(c, GF_EINVAL, "mu is not finite");
  gf_status st = check_ready(c);
  if (st) return st;
  if (!c->use_graph || c->occ_calls == 0) {
    // ordinary enqueue (also the warm-up of graph mode: scratch, autotuner)
    ++c->occ_calls;
    GF_CU(cudaStreamSynchronize(c->stream));  // hp_mu is about to be rewritten
    for (int s2 = 0; s2 < c->n_sys; ++s2) c->hp_mu()[s2] = mu[s2];
    st = enqueue_occupation(c);
    if (st) return st;
    return finish_occupation(c, c->stream, n_out, dn_out);
  }
  // graph mode: E_inf and the low-rank eigenbasis outside the graph (inputs may
  // have changed), then replay
  GF_CU(cudaStreamSynchronize(c->stream));
  st = ensure_einf(c);
  if (st) return st;
  if (c->lowrank && c->lr_dirty) {
    GF_CU(cudaMemsetAsync(c->status.p, 0, sizeof(int), c->stream));
    st = ensure_lr(c);
    if (st) return st;
    st = sync_and_check(c);
    if (st) return st;
  }
  for (int s2 = 0; s2 < c->n_sys; ++s2) c->hp_mu()[s2] = mu[s2];
  if (!c->occ_exec) {
    GF_CU(cudaStreamSynchronize(c->stream));
    const cudaStream_t user = c->stream;
    c->stream = c->cap_stream;
    const int64_t l0 = c->last_launches, p0 = c->last_points;
    const double f0 = c->last_flops;
    c->ev_used = 0;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      c->capturing = true;
      try {
        st = enqueue_occupation(c);
      } catch (...) {
        // end the capture and give the caller's stream back before the status is reported
        c->capturing = false;
        if (cudaStreamEndCapture(c->stream, &graph) == cudaSuccess && graph) cudaGraphDestroy(graph);
        c->stream = user;
        throw;
      }
      c->capturing = false;
      cudaError_t e2 = cudaStreamEndCapture(c->stream, &graph);
      if (st == GF_OK && e2 != cudaSuccess) e = e2;
    }
    c->stream = user;
    if (st) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return fail(c, GF_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&c->occ_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      c->occ_exec = nullptr;
      return fail(c, GF_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    c->occ_launches = c->last_launches - l0;
    c->occ_points = c->last_points - p0;
    c->occ_flops = c->last_flops - f0;
    c->last_launches = l0;
    c->last_points = p0;
    c->last_flops = f0;
  }
  GF_CU(cudaEventRecord(c->ev_user, c->stream));
  GF_CU(cudaStreamWaitEvent(c->cap_stream, c->ev_user, 0));
  reserve_events(c, 2);
  while (c->ev.size() < 2) {
    cudaEvent_t e;
    GF_CU(cudaEventCreate(&e));
    c->ev.push_back(e);
  }
  GF_CU(cudaEventRecord(c->ev[0], c->cap_stream));
  GF_CU(cudaGraphLaunch(c->occ_exec, c->cap_stream));
  GF_CU(cudaEventRecord(c->ev[1], c->cap_stream));
  c->ev_used = 2;
  c->last_launches += c->occ_launches;
  c->last_points += c->occ_points;
  c->last_flops += c->occ_flops;
  return finish_occupation(c, c->cap_stream, n_out, dn_out);
}

}  // namespace

namespace {

// Fills a new context from its descriptor and allocates its device workspace.  It never
// frees the context: gf_create discards it on a failed status and on a C++ exception alike.
gf_status init_ctx(gf_ctx* c, const gf_desc* d) {
  auto bad = [](const char* m) {
    gf::set_global_error(m);
    return GF_EINVAL;
  };
  c->n_sys = d->n_systems;
  c->n_k = d->n_k;
  c->n_iw = d->n_iw;
  c->precision = d->precision;
  c->in_dtype = d->input_dtype;
  c->tail_order = d->tail_order;
  c->device = d->device;
  c->stream = static_cast<cudaStream_t>(d->stream);
  c->use_graph = (d->flags & GF_FLAG_GRAPH) != 0;
  c->lowrank = (d->flags & GF_FLAG_LOWRANK) != 0;
  c->nb.resize(c->n_k);
  c->ksys.resize(c->n_k);
  for (int k = 0; k < c->n_k; ++k) {
    c->nb[k] = d->nb ? d->nb[k] : d->nb_uniform;
    c->ksys[k] = d->k_system ? d->k_system[k] : 0;
    if (c->nb[k] < 1) return bad("every N_b(k) must be >= 1");
    if (c->ksys[k] < 0 || c->ksys[k] >= c->n_sys) return bad("k_system out of range");
    if (k > 0 && c->ksys[k] < c->ksys[k - 1]) return bad("k_system must be non-decreasing");
  }
  c->msys.assign(d->m_system, d->m_system + c->n_sys);
  c->beta.assign(d->beta, d->beta + c->n_sys);
  for (int s = 0; s < c->n_sys; ++s) {
    if (c->msys[s] < 1) return bad("every m must be >= 1");
    if (!(c->beta[s] > 0.0) || !std::isfinite(c->beta[s])) return bad("beta must be > 0");
  }
  // systems, k ranges and weights
  c->sinfo.resize(c->n_sys);
  std::vector<int> count(c->n_sys, 0);
  for (int k = 0; k < c->n_k; ++k) count[c->ksys[k]]++;
  int64_t offSig = 0, offSinf = 0;
  int k0 = 0;
  for (int s = 0; s < c->n_sys; ++s) {
    if (count[s] == 0) return bad("a system has no k-points");
    SInfo& si = c->sinfo[s];
    si.m = c->msys[s];
    si.k0 = k0;
    si.k1 = k0 + count[s];
    k0 = si.k1;
    si.pad = 0;
    si.beta = c->beta[s];
    si.tailc = gf::tail_coefficient(si.beta, c->n_iw, c->tail_order);
    si.offSig = offSig;
    si.offSinf = offSinf;
    offSig += (int64_t)c->n_iw * si.m * si.m;
    offSinf += (int64_t)si.m * si.m;
    c->mmax = std::max(c->mmax, si.m);
  }
  c->totSig = offSig;
  c->totSinf = offSinf;
  c->kinfo.resize(c->n_k);
  c->wk.resize(c->n_k);
  c->offD.resize(c->n_k);
  int64_t offH = 0, offP = 0, offD = 0;
  for (int k = 0; k < c->n_k; ++k) {
    KInfo& ki = c->kinfo[k];
    ki.nb = c->nb[k];
    ki.sys = c->ksys[k];
    ki.offH = offH;
    ki.offP = offP;
    const SInfo& si = c->sinfo[ki.sys];
    ki.w = d->k_weight ? d->k_weight[k] : 1.0 / (si.k1 - si.k0);
    if (!std::isfinite(ki.w)) return bad("k_weight is not finite");
    c->wk[k] = ki.w;
    c->offD[k] = offD;
    offH += (int64_t)ki.nb * ki.nb;
    offP += (int64_t)si.m * ki.nb;
    offD += ki.nb;
    c->nbmax = std::max(c->nbmax, ki.nb);
  }
  c->totH = offH;
  c->totP = offP;
  c->totNb = offD;
  c->sys_dtype.resize(c->n_sys);
  c->sysH.resize(c->n_sys + 1);
  c->sysD.resize(c->n_sys + 1);
  c->sysP.resize(c->n_sys + 1);
  c->sysSig.resize(c->n_sys + 1);
  c->sysSinf.resize(c->n_sys + 1);
  for (int s = 0; s < c->n_sys; ++s) {
    const SInfo& si = c->sinfo[s];
    c->sys_dtype[s] = d->system_dtype ? d->system_dtype[s] : d->input_dtype;
    c->sysH[s] = c->kinfo[si.k0].offH;
    c->sysD[s] = c->offD[si.k0];
    c->sysP[s] = c->kinfo[si.k0].offP;
    c->sysSig[s] = si.offSig;
    c->sysSinf[s] = si.offSinf;
  }
  c->sysH[c->n_sys] = c->totH;
  c->sysD[c->n_sys] = c->totNb;
  c->sysP[c->n_sys] = c->totP;
  c->sysSig[c->n_sys] = c->totSig;
  c->sysSinf[c->n_sys] = c->totSinf;
  for (int k = 0; k < c->n_k; ++k) {
    const int bk = gf_bucket(c->nb[k]);
    c->bucket_nbmax[bk] = std::max(c->bucket_nbmax[bk], c->nb[k]);
  }

  // device
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    gf::set_global_error("no CUDA device");
    return GF_ECUDA;
  }
  if (c->device < 0 || c->device >= ndev) return bad("device ordinal out of range");
  c->device_checked = true;
  DeviceGuard guard(c->device);
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
  cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  // the k-reductions keep one slot of n_iw * mmax^2 complex numbers per k-group in gq,
  // batched within a quarter of the free device memory and at most 32 GiB
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    free_b = (size_t)32 << 30;
  }
  size_t budget = std::min<size_t>((size_t)32 << 30, std::max<size_t>(free_b / 4, (size_t)1 << 28));
  if (const char* env = std::getenv("GF_GQ_BUDGET_MB")) budget = (size_t)std::atoll(env) << 20;
  c->gq_budget = budget;
  const size_t per_group = sizeof(double2) * (size_t)c->n_iw * c->mmax * c->mmax;
  // chunk width: about 40 items per resident CTA in each window bucket's launch
  // (resident CTAs: the larger of the two matrix placements of the point kernel)
  int bps = 1;
  for (int in_smem = 0; in_smem <= 1; ++in_smem) {
    const size_t smem = gf::point_fp64_smem(c->nbmax, c->mmax, gf::kOcc, in_smem);
    if (smem <= (size_t)c->smem_optin - 1024)
      bps = std::max(bps, (c->precision != GF_PREC_FP64) ? gf::point_df64_blocks_per_sm(smem)
                                                          : gf::point_fp64_blocks_per_sm(smem));
  }
  int n_buckets = 0;
  for (int b = 0; b < kNumBuckets; ++b) n_buckets += c->bucket_nbmax[b] > 0;
  const double resident = (double)c->sm_count * bps;
  const double want = (double)c->n_k * c->n_iw / (40.0 * resident * std::max(1, n_buckets));
  c->chunk_w = (int)std::min<double>(c->n_iw, std::max(4.0, std::ceil(want)));
  c->n_chunks = (c->n_iw + c->chunk_w - 1) / c->chunk_w;
  // Work items.  Modes without a k-reduction: one item per (k, chunk), all in one list
  // sorted by decreasing window (one launch per window bucket).  Modes with a k-reduction:
  // the k-points of each system and window bucket, in increasing k, form groups of kg;
  // one item per (group, chunk) sums its k-points into one slot per (group, frequency),
  // so the scratch holds n_iw mmax^2 numbers per group instead of per k-point.  kg keeps
  // about 8 items per resident CTA.
  // groups share a window bucket; order by the window of their first k-point
  auto by_window = [&](const Item& a, const Item& b) { return c->nb[c->kperm[a.k]] > c->nb[c->kperm[b.k]]; };
  c->kg = (int)std::max(1.0, std::min((double)gf::kMaxKGroup, std::floor((double)c->n_k * c->n_chunks / (8.0 * resident))));
  c->kperm.clear();
  c->group_k0.clear();
  c->group_nk.clear();
  c->sys_g0.assign(c->n_sys, 0);
  c->sys_g1.assign(c->n_sys, 0);
  for (int s = 0; s < c->n_sys; ++s) {
    c->sys_g0[s] = (int)c->group_k0.size();
    for (int b = kNumBuckets - 1; b >= 0; --b) {
      int in_group = 0;
      for (int k = c->sinfo[s].k0; k < c->sinfo[s].k1; ++k) {
        if (gf_bucket(c->nb[k]) != b) continue;
        if (in_group == 0) {
          c->group_k0.push_back((int)c->kperm.size());
          c->group_nk.push_back(0);
        }
        c->kperm.push_back(k);
        ++c->group_nk.back();
        if (++in_group == c->kg) in_group = 0;
      }
    }
    c->sys_g1[s] = (int)c->group_k0.size();
  }
  c->n_groups = (int)c->group_k0.size();
  const int gpb = (int)std::max<size_t>(1, std::min<size_t>(c->n_groups, budget / per_group));
  c->items.clear();
  c->batch_g0.clear();
  c->batch_item0.clear();
  for (int gb = 0; gb < c->n_groups; gb += gpb) {
    const int ge = std::min(c->n_groups, gb + gpb);
    c->batch_g0.push_back(gb);
    c->batch_item0.push_back((int)c->items.size());
    std::vector<Item> its;
    for (int g = gb; g < ge; ++g)
      for (int ch = 0; ch < c->n_chunks; ++ch)
        its.push_back(Item{c->group_k0[g], ch * c->chunk_w, std::min(c->n_iw, (ch + 1) * c->chunk_w), ch,
                           c->group_nk[g], g});
    // most expensive first (N_b^3), stable in (group, chunk)
    std::stable_sort(its.begin(), its.end(), by_window);
    c->items.insert(c->items.end(), its.begin(), its.end());
  }
  c->batch_g0.push_back(c->n_groups);
  c->batch_item0.push_back((int)c->items.size());
  {
    std::vector<Item> all;
    for (int k = 0; k < c->n_k; ++k)
      for (int ch = 0; ch < c->n_chunks; ++ch)
        all.push_back(Item{k, ch * c->chunk_w, std::min(c->n_iw, (ch + 1) * c->chunk_w), ch, 1, k});
    std::stable_sort(all.begin(), all.end(), [&](const Item& a, const Item& b) { return c->nb[a.k] > c->nb[b.k]; });
    c->all_item0 = (int)c->items.size();
    c->n_items_all = (int)all.size();
    c->items.insert(c->items.end(), all.begin(), all.end());
  }

  auto alloc_all = [&]() -> cudaError_t {
    cudaError_t e;
    if ((e = ensure(c->H, sizeof(double2) * c->totH))) return e;
    if ((e = ensure(c->Einf, sizeof(double2) * c->totH))) return e;
    if ((e = ensure(c->P, sizeof(double2) * c->totP))) return e;
    if ((e = ensure(c->Sig, sizeof(double2) * c->totSig))) return e;
    if ((e = ensure(c->gacc, sizeof(double2) * c->totSig))) return e;
    if ((e = ensure(c->Sinf, sizeof(double2) * c->totSinf))) return e;
    if (c->precision != GF_PREC_FP64) {
      if ((e = ensure(c->Hd, sizeof(float4) * c->totH))) return e;
      if ((e = ensure(c->Pd, sizeof(float4) * c->totP))) return e;
      if ((e = ensure(c->Sd, sizeof(float4) * c->totSig))) return e;
    }
    if (c->precision == GF_PREC_MIXED) {
      if ((e = ensure(c->Hs, sizeof(float2) * c->totH))) return e;
      if ((e = ensure(c->Ps, sizeof(float2) * c->totP))) return e;
      if ((e = ensure(c->Ss, sizeof(float2) * c->totSig))) return e;
    }
    if ((e = ensure(c->trHE, sizeof(double) * c->n_k))) return e;
    if ((e = ensure(c->kN, sizeof(double) * c->n_k))) return e;
    if ((e = ensure(c->kdN, sizeof(double) * c->n_k))) return e;
    if ((e = ensure(c->kNc, sizeof(double) * c->n_k))) return e;
    if ((e = ensure(c->kinfo_d, sizeof(KInfo) * c->n_k))) return e;
    if ((e = ensure(c->sinfo_d, sizeof(SInfo) * c->n_sys))) return e;
    if ((e = ensure(c->items_d, sizeof(Item) * c->items.size()))) return e;
    if ((e = ensure(c->kperm_d, sizeof(int) * c->kperm.size()))) return e;
    if ((e = ensure(c->sysg_d, sizeof(int) * 2 * c->n_sys))) return e;
    if ((e = ensure(c->offD_d, sizeof(int64_t) * c->n_k))) return e;
    if ((e = ensure(c->mu, sizeof(double) * c->n_sys))) return e;
    if ((e = ensure(c->nbar, sizeof(double) * c->n_sys))) return e;
    if ((e = ensure(c->mubar_sys, sizeof(double) * c->n_sys))) return e;
    if ((e = ensure(c->sysout2, sizeof(double) * 2 * c->n_sys))) return e;
    if ((e = ensure(c->sysout, sizeof(double) * 2 * c->n_sys))) return e;
    if ((e = ensure(c->status, sizeof(int)))) return e;
    if ((e = ensure(c->queue, sizeof(int)))) return e;
    if ((e = cudaMallocHost(&c->hpin, sizeof(double) * (8 + 7 * (size_t)c->n_sys)))) return e;
    if ((e = cudaMemcpyAsync(c->kinfo_d.p, c->kinfo.data(), sizeof(KInfo) * c->n_k,
                             cudaMemcpyHostToDevice, c->stream)))
      return e;
    if ((e = cudaMemcpyAsync(c->sinfo_d.p, c->sinfo.data(), sizeof(SInfo) * c->n_sys,
                             cudaMemcpyHostToDevice, c->stream)))
      return e;
    if ((e = cudaMemcpyAsync(c->items_d.p, c->items.data(), sizeof(Item) * c->items.size(),
                             cudaMemcpyHostToDevice, c->stream)))
      return e;
    if ((e = cudaMemcpyAsync(c->kperm_d.p, c->kperm.data(), sizeof(int) * c->kperm.size(),
                             cudaMemcpyHostToDevice, c->stream)))
      return e;
    std::vector<int> sysg(c->sys_g0);
    sysg.insert(sysg.end(), c->sys_g1.begin(), c->sys_g1.end());
    if ((e = cudaMemcpyAsync(c->sysg_d.p, sysg.data(), sizeof(int) * 2 * c->n_sys,
                             cudaMemcpyHostToDevice, c->stream)))
      return e;
    if ((e = cudaMemcpyAsync(c->offD_d.p, c->offD.data(), sizeof(int64_t) * c->n_k,
                             cudaMemcpyHostToDevice, c->stream)))
      return e;
    if ((e = cudaMemsetAsync(c->status.p, 0, sizeof(int), c->stream))) return e;
    if (c->use_graph) {
      if ((e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking))) return e;
      if ((e = cudaEventCreateWithFlags(&c->ev_user, cudaEventDisableTiming))) return e;
    }
    return cudaStreamSynchronize(c->stream);
  };
  cudaError_t e = alloc_all();
  if (e != cudaSuccess) {
    char msg[160];
    std::snprintf(msg, sizeof(msg), "device setup failed: %s", cudaGetErrorString(e));
    gf::set_global_error(msg);
    return e == cudaErrorMemoryAllocation ? GF_ENOMEM : GF_ECUDA;
  }
  return GF_OK;
}

// Frees a context that gf_create does not hand out: by gf_destroy once its device ordinal
// has been checked, before that by a plain delete, so that no CUDA call is made on an
// invalid device and no CUDA error is left behind.
void discard_ctx(gf_ctx* c) noexcept {
  if (c->device_checked)
    gf_destroy(c);
  else
    delete c;
}

}  // namespace

extern "C" {

gf_status gf_create(gf_ctx** out, const gf_desc* d) try {
  gf::set_global_error("");
  if (!out) {
    gf::set_global_error("out is NULL");
    return GF_EINVAL;
  }
  *out = nullptr;
  auto bad = [](const char* m) {
    gf::set_global_error(m);
    return GF_EINVAL;
  };
  if (!d) return bad("desc is NULL");
  if (d->n_systems < 1) return bad("n_systems must be >= 1");
  if (d->n_k < 1) return bad("n_k must be >= 1");
  if (d->n_iw < 1) return bad("n_iw must be >= 1");
  if (!d->m_system) return bad("m_system is NULL");
  if (!d->beta) return bad("beta is NULL");
  if (!d->nb && d->nb_uniform < 1) return bad("nb is NULL and nb_uniform < 1");
  if (d->precision != GF_PREC_FP64 && d->precision != GF_PREC_MIXED && d->precision != GF_PREC_PAIR)
    return bad("bad precision");
  if (d->input_dtype != GF_C128 && d->input_dtype != GF_C64) return bad("bad input_dtype");
  if (d->system_dtype)
    for (int s = 0; s < d->n_systems; ++s)
      if (d->system_dtype[s] != GF_C128 && d->system_dtype[s] != GF_C64) return bad("bad system_dtype");
  if (d->tail_order != 1 && d->tail_order != 2) return bad("tail_order must be 1 or 2");
  gf_ctx* c = new (std::nothrow) gf_ctx();
  if (!c) {
    gf::set_global_error("host allocation failed");
    return GF_ENOMEM;
  }
  gf_status st;
  try {
    st = init_ctx(c, d);
  } catch (...) {
    discard_ctx(c);
    throw;
  }
  if (st != GF_OK) {
    discard_ctx(c);
    return st;
  }
  *out = c;
  return GF_OK;
} catch (...) {
  return caught(nullptr);
}

gf_status gf_destroy(gf_ctx* c) {
  if (!c) return GF_OK;
  DeviceGuard guard(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  DevBuf* bufs[] = {&c->H, &c->P, &c->Sig, &c->Sinf, &c->Einf, &c->trHE, &c->kinfo_d, &c->sinfo_d,
                    &c->items_d, &c->offD_d, &c->mu, &c->nbar, &c->gbar, &c->status, &c->queue,
                    &c->stage, &c->occ_part, &c->rho_part, &c->rho_out, &c->gq, &c->kN, &c->kdN,
                    &c->kNc, &c->sysout, &c->a_scratch, &c->mubar_part, &c->mubar_sys, &c->gacc,
                    &c->sysout2, &c->Hd, &c->Pd, &c->Sd, &c->Gbd, &c->poles, &c->Vp,
                    &c->Sinf_p, &c->pinfo_d, &c->eoff_d, &c->phioff_d, &c->eout, &c->phiout,
                    &c->pole_ws, &c->lr_eps, &c->lr_U, &c->lr_Pt, &c->lr_T, &c->lr_ws,
                    &c->eimp, &c->eimp_part, &c->gl_in, &c->delta, &c->wraw, &c->vdc,
                    &c->wbout, &c->kHks, &c->kEps, &c->eps_grid, &c->dos, &c->pdos, &c->pdos_off,
                    &c->pole_part, &c->pole_vs, &c->pole_es, &c->voff_d, &c->mu_prev};
  for (DevBuf* b : bufs) release(*b);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  if (c->occ_exec) cudaGraphExecDestroy(c->occ_exec);
  if (c->ev_user) cudaEventDestroy(c->ev_user);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->hpin) cudaFreeHost(c->hpin);
  delete c;
  return GF_OK;
}

gf_status gf_set_hamiltonian(gf_ctx* c, const void* h, int32_t is_diagonal) try {
  NvtxRange nvtx_range_("gf_set_hamiltonian");
  if (!c) return GF_EINVAL;
  if (!h) return fail(c, GF_EINVAL, "h_ptr is NULL");
  DeviceGuard guard(c->device);
  if (is_diagonal) {
    GF_CU(ensure(c->stage, 0));
    DevBuf diag;
    gf_status st = GF_OK;
    cudaError_t e = ensure(diag, sizeof(double2) * c->totNb);
    if (e != cudaSuccess) return fail(c, GF_ENOMEM, "allocation of the diagonal staging failed");
    st = load_complex(c, h, c->sysD, diag.as<double2>());
    if (st == GF_OK) {
      e = gf::launch_diag_to_dense(c->kinfo_d.as<KInfo>(), diag.as<double2>(), c->offD_d.as<int64_t>(),
                                   c->n_k, c->H.as<double2>(), c->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
      if (e != cudaSuccess) st = fail(c, GF_ECUDA, std::string("diagonal H: ") + cudaGetErrorString(e));
    }
    release(diag);
    if (st) return st;
  } else {
    gf_status st = load_complex(c, h, c->sysH, c->H.as<double2>());
    if (st) return st;
    GF_CU(cudaStreamSynchronize(c->stream));
  }
  if (c->precision != GF_PREC_FP64) {
    gf_status st = derive_f32(c, c->H, c->Hd, &c->Hs, c->totH);
    if (st) return st;
    GF_CU(cudaStreamSynchronize(c->stream));
  }
  c->have_H = true;
  c->lr_dirty = true;
  c->einf_dirty = true;
  return GF_OK;
} catch (...) {
  return caught(c);
}

gf_status gf_set_projectors(gf_ctx* c, const void* p) try {
  NvtxRange nvtx_range_("gf_set_projectors");
  if (!c) return GF_EINVAL;
  if (!p) return fail(c, GF_EINVAL, "p_ptr is NULL");
  DeviceGuard guard(c->device);
  gf_status st = load_complex(c, p, c->sysP, c->P.as<double2>());
  if (st) return st;
  st = derive_f32(c, c->P, c->Pd, &c->Ps, c->totP);
  if (st) return st;
  GF_CU(cudaStreamSynchronize(c->stream));
  c->have_P = true;
  c->lr_dirty = true;
  c->einf_dirty = true;
  return GF_OK;
} catch (...) {
  return caught(c);
}

gf_status gf_set_sigma(gf_ctx* c, const void* sig, const void* sinf) try {
  NvtxRange nvtx_range_("gf_set_sigma");
  if (!c) return GF_EINVAL;
  if (!sig || !sinf) return fail(c, GF_EINVAL, "sigma_iw_ptr or sigma_inf_ptr is NULL");
  DeviceGuard guard(c->device);
  gf_status st = load_complex(c, sig, c->sysSig, c->Sig.as<double2>());
  if (st) return st;
  st = load_complex(c, sinf, c->sysSinf, c->Sinf.as<double2>());
  if (st) return st;
  st = derive_f32(c, c->Sig, c->Sd, &c->Ss, c->totSig);
  if (st) return st;
  GF_CU(cudaStreamSynchronize(c->stream));
  c->have_S = true;
  c->einf_dirty = true;
  return GF_OK;
} catch (...) {
  return caught(c);
}

gf_status gf_occupation(gf_ctx* c, const double* mu, double* n_out, double* dn_out) try {
  NvtxRange nvtx_range_("gf_occupation");
  if (!c) return GF_EINVAL;
  if (!n_out) return fail(c, GF_EINVAL, "n_out is NULL");
  DeviceGuard guard(c->device);
  reset_stats(c);
  return occupation_impl(c, mu, n_out, dn_out);
} catch (...) {
  return caught(c);
}

gf_status gf_find_mu(gf_ctx* c, const double* n_target, double tol, int32_t max_iter,
                     double* mu_inout, int32_t* iters_out) try {
  NvtxRange nvtx_range_("gf_find_mu");
  if (!c) return GF_EINVAL;
  DeviceGuard guard(c->device);
  reset_stats(c);
  return newton_mu(c, n_target, tol, max_iter, mu_inout, iters_out,
                   [c](const double* mu, double* n, double* dn) {
                     return occupation_impl(c, mu, n, dn);  // stats accumulate
                   });
} catch (...) {
  return caught(c);
}

gf_status gf_density_matrix(gf_ctx* c, const double* mu, void* rho_out, double* n_corr_out) try {
  NvtxRange nvtx_range_("gf_density_matrix");
  if (!c) return GF_EINVAL;
  DeviceGuard guard(c->device);
  reset_stats(c);
  gf_status st = upload_mu(c, mu);
  if (st) return st;
  st = run_points(c, gf::kRho);
  if (st) return st;
  int nch = 0;
  st = rho_partials(c, &nch);
  if (st) return st;
  GF_CU(ensure(c->rho_out, sizeof(double2) * c->totH));
  GF_CU(gf::launch_rho_finalize(c->kinfo_d.as<KInfo>(), c->sinfo_d.as<SInfo>(), c->H.as<double2>(),
                                c->Einf.as<double2>(), c->P.as<double2>(), c->mu.as<double>(),
                                c->rho_part.as<double2>(), c->totH, nch, c->n_k,
                                c->rho_out.as<double2>(), c->kN.as<double>(), c->kNc.as<double>(),
                                c->stream));
  GF_CU(gf::launch_sys_reduce(c->kinfo_d.as<KInfo>(), c->sinfo_d.as<SInfo>(), c->n_sys,
                              c->kNc.as<double>(), c->kN.as<double>(), c->sysout.as<double>(),
                              c->stream));
  c->last_launches += 2;
  if (rho_out)
    GF_CU(cudaMemcpyAsync(rho_out, c->rho_out.p, sizeof(double2) * c->totH, cudaMemcpyDefault,
                          c->stream));
  GF_CU(cudaMemcpyAsync(c->hp_sys(), c->sysout.p, sizeof(double) * 2 * c->n_sys,
                        cudaMemcpyDeviceToHost, c->stream));
  st = sync_and_check(c);
  if (st) return st;
  if (n_corr_out)
    for (int s = 0; s < c->n_sys; ++s) n_corr_out[s] = c->hp_sys()[2 * s];
  return GF_OK;
} catch (...) {
  return caught(c);
}

gf_status gf_local(gf_ctx* c, const double* mu, void* gloc_out) try {
  NvtxRange nvtx_range_("gf_local");
  if (!c) return GF_EINVAL;
  if (!gloc_out) return fail(c, GF_EINVAL, "gloc_out_ptr is NULL");
  DeviceGuard guard(c->device);
  reset_stats(c);
  gf_status st = upload_mu(c, mu);
  if (st) return st;
  st = run_points(c, gf::kGloc);
  if (st) return st;
  GF_CU(cudaMemcpyAsync(gloc_out, c->gacc.p, sizeof(double2) * c->totSig, cudaMemcpyDefault,
                        c->stream));
  return sync_and_check(c);
} catch (...) {
  return caught(c);
}

gf_status gf_evaluate(gf_ctx* c, const double* mu, void* gloc_out, void* rho_out, double* n_out,
                      double* dn_out, double* n_corr_out) try {
  NvtxRange nvtx_range_("gf_evaluate");
  if (!c) return GF_EINVAL;
  const int mode = (gloc_out ? gf::kGloc : 0) | ((rho_out || n_corr_out) ? gf::kRho : 0) |
                   ((n_out || dn_out) ? gf::kOcc : 0);
  if (!mode) return fail(c, GF_EINVAL, "every output of gf_evaluate is NULL");
  DeviceGuard guard(c->device);
  reset_stats(c);
  gf_status st = upload_mu(c, mu);
  if (st) return st;
  st = run_points(c, mode);
  if (st) return st;
  if (mode & gf::kOcc) {
    GF_CU(gf::launch_occ_finalize(c->kinfo_d.as<KInfo>(), c->sinfo_d.as<SInfo>(),
                                  c->trHE.as<double>(), c->mu.as<double>(), c->occ_part.as<double>(),
                                  c->n_chunks, c->n_k, c->kN.as<double>(), c->kdN.as<double>(),
                                  c->stream));
    GF_CU(gf::launch_sys_reduce(c->kinfo_d.as<KInfo>(), c->sinfo_d.as<SInfo>(), c->n_sys,
                                c->kN.as<double>(), c->kdN.as<double>(), c->sysout.as<double>(),
                                c->stream));
    c->last_launches += 2;
    GF_CU(cudaMemcpyAsync(c->hp_sys(), c->sysout.p, sizeof(double) * 2 * c->n_sys,
                          cudaMemcpyDeviceToHost, c->stream));
  }
  if (mode & gf::kRho) {
    int nch = 0;
    st = rho_partials(c, &nch);
    if (st) return st;
    GF_CU(ensure(c->rho_out, sizeof(double2) * c->totH));
    GF_CU(gf::launch_rho_finalize(c->kinfo_d.as<KInfo>(), c->sinfo_d.as<SInfo>(), c->H.as<double2>(),
                                  c->Einf.as<double2>(), c->P.as<double2>(), c->mu.as<double>(),
                                  c->rho_part.as<double2>(), c->totH, nch, c->n_k,
                                  c->rho_out.as<double2>(), c->kN.as<double>(), c->kNc.as<double>(),
                                  c->stream));
    GF_CU(gf::launch_sys_reduce(c->kinfo_d.as<KInfo>(), c->sinfo_d.as<SInfo>(), c->n_sys,
                                c->kNc.as<double>(), c->kN.as<double>(), c->sysout2.as<double>(),
                                c->stream));
    c->last_launches += 2;
    GF_CU(cudaMemcpyAsync(c->hp_sys2(), c->sysout2.p, sizeof(double) * 2 * c->n_sys,
                          cudaMemcpyDeviceToHost, c->stream));
    if (rho_out)
      GF_CU(cudaMemcpyAsync(rho_out, c->rho_out.p, sizeof(double2) * c->totH, cudaMemcpyDefault,
                            c->stream));
  }
  if (gloc_out)
    GF_CU(cudaMemcpyAsync(gloc_out, c->gacc.p, sizeof(double2) * c->totSig, cudaMemcpyDefault,
                          c->stream));
  st = sync_and_check(c);
  if (st) return st;
  for (int s = 0; s < c->n_sys; ++s) {
    if (n_out) n_out[s] = c->hp_sys()[2 * s];
    if (dn_out) dn_out[s] = c->hp_sys()[2 * s + 1];
  }
  if (n_corr_out)
    for (int s = 0; s < c->n_sys; ++s) n_corr_out[s] = c->hp_sys2()[2 * s];
  return GF_OK;
} catch (...) {
  return caught(c);
}

gf_status gf_backward(gf_ctx* c, const double* mu, const void* gbar, const double* nbar,
                      void* sbar_out, double* mubar_out) try {
  NvtxRange nvtx_range_("gf_backward");
  if (!c) return GF_EINVAL;
  if (!sbar_out || !mubar_out) return fail(c, GF_EINVAL, "sigma_bar_out_ptr or mu_bar_out is NULL");
  DeviceGuard guard(c->device);
  reset_stats(c);
  gf_status st = upload_mu(c, mu);
  if (st) return st;
  bool any_nbar = false;
  for (int s = 0; s < c->n_sys; ++s) {
    const double v = nbar ? nbar[s] : 0.0;
    if (!std::isfinite(v)) return fail(c, GF_EINVAL, "n_bar is not finite");
    c->hp_nbar()[s] = v;
    any_nbar = any_nbar || v != 0.0;
  }
  GF_CU(cudaMemcpyAsync(c->nbar.p, c->hp_nbar(), sizeof(double) * c->n_sys, cudaMemcpyHostToDevice,
                        c->stream));
  c->have_gbar_for_call = (gbar != nullptr);
  if (gbar) {
    GF_CU(ensure(c->gbar, sizeof(double2) * c->totSig));
    GF_CU(cudaMemcpyAsync(c->gbar.p, gbar, sizeof(double2) * c->totSig, cudaMemcpyDefault, c->stream));
    if (c->precision != GF_PREC_FP64) {
      GF_CU(ensure(c->Gbd, sizeof(float4) * c->totSig));
      GF_CU(gf::launch_split_df64(c->gbar.as<double2>(), c->Gbd.as<float4>(), c->totSig, c->stream));
    }
  }
  const int mode = gf::kAdj | (any_nbar ? gf::kOcc : 0);
  st = run_points(c, mode);
  if (st) return st;
  GF_CU(gf::launch_mubar_reduce(c->kinfo_d.as<KInfo>(), c->sinfo_d.as<SInfo>(), c->n_sys,
                                c->n_chunks, c->mubar_part.as<double>(), c->mubar_sys.as<double>(),
                                c->stream));
  c->last_launches += 1;
  if (any_nbar) {
    GF_CU(gf::launch_occ_finalize(c->kinfo_d.as<KInfo>(), c->sinfo_d.as<SInfo>(),
                                  c->trHE.as<double>(), c->mu.as<double>(), c->occ_part.as<double>(),
                                  c->n_chunks, c->n_k, c->kN.as<double>(), c->kdN.as<double>(),
                                  c->stream));
    GF_CU(gf::launch_sys_reduce(c->kinfo_d.as<KInfo>(), c->sinfo_d.as<SInfo>(), c->n_sys,
                                c->kN.as<double>(), c->kdN.as<double>(), c->sysout.as<double>(),
                                c->stream));
    c->last_launches += 2;
    GF_CU(cudaMemcpyAsync(c->hp_sys(), c->sysout.p, sizeof(double) * 2 * c->n_sys,
                          cudaMemcpyDeviceToHost, c->stream));
  }
  GF_CU(cudaMemcpyAsync(c->hp_mubar(), c->mubar_sys.p, sizeof(double) * c->n_sys,
                        cudaMemcpyDeviceToHost, c->stream));
  GF_CU(cudaMemcpyAsync(sbar_out, c->gacc.p, sizeof(double2) * c->totSig, cudaMemcpyDefault,
                        c->stream));
  st = sync_and_check(c);
  if (st) return st;
  for (int s = 0; s < c->n_sys; ++s) {
    const double dn = any_nbar ? c->hp_sys()[2 * s + 1] : 0.0;
    mubar_out[s] = c->hp_nbar()[s] * dn + c->hp_mubar()[s];
  }
  return GF_OK;
} catch (...) {
  return caught(c);
}

const char* gf_tuning_log(const gf_ctx* c) {
  if (!c) return "";
  return c->tune_log.c_str();
}

const char* gf_last_error(const gf_ctx* c) {
  if (!c) return g_create_error.c_str();
  return c->err.c_str();
}

gf_status gf_last_stats(const gf_ctx* c, int64_t* launches, int64_t* points, double* kernel_ms,
                        double* flops) {
  if (!c) return GF_EINVAL;
  if (launches) *launches = c->last_launches;
  if (points) *points = c->last_points;
  if (kernel_ms) *kernel_ms = c->last_kernel_ms;
  if (flops) *flops = c->last_flops;
  return GF_OK;
}

}  // extern "C"
