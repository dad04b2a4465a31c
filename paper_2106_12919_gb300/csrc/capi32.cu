// C ABI of the FP32 form: the same orchestration as pic_step (capi.cu) on float
// arrays.  Spectra and nodal work arrays live in the context buffers (sized for
// FP64, so an FP32 context uses the first half of each).
#include "pic_internal.cuh"

namespace {

#define PIC_TRY32(x)               \
  do {                             \
    pic_status s_ = (x);           \
    if (s_ != PIC_OK) return s_;   \
  } while (0)

#define PIC_NEED_FP32(ctx)                                                                    \
  do {                                                                                        \
    if (!(ctx)) return PIC_ERR_ARG;                                                           \
    if ((ctx)->precision != PIC_FP32)                                                         \
      return pic_set_error((ctx), PIC_ERR_ARG, "FP32 entry point on an FP64 context");        \
  } while (0)

template <class P>
bool nonnull(P const* a, int n) {
  if (!a) return false;
  for (int i = 0; i < n; ++i)
    if (!a[i]) return false;
  return true;
}

pic_status check_species32(pic_ctx* ctx, const pic_species32* sp, int n_species) {
  if (n_species < 0 || (n_species > 0 && sp == nullptr)) return pic_set_error(ctx, PIC_ERR_ARG, "species array");
  for (int s = 0; s < n_species; ++s) {
    const pic_species32& p = sp[s];
    if (p.n < 0) return pic_set_error(ctx, PIC_ERR_ARG, "species %d: negative count", s);
    if (p.n > 0 && (!p.cell || !p.fx || !p.fy || !p.fz || !p.ux || !p.uy || !p.uz || !p.w))
      return pic_set_error(ctx, PIC_ERR_ARG, "species %d: null array", s);
    if (!(p.m > 0.0)) return pic_set_error(ctx, PIC_ERR_ARG, "species %d: mass must be > 0", s);
    if (p.n > ((int64_t)1 << 31) - 1)
      return pic_set_error(ctx, PIC_ERR_CAPACITY, "species %d: more than 2^31-1 particles", s);
  }
  return PIC_OK;
}

const int kKindEB[6] = {0, 1, 2, 3, 4, 5};
const int kKindJ[3] = {6, 7, 8};

inline float2* f2(double2* p) { return reinterpret_cast<float2*>(p); }
inline float* f1(double* p) { return reinterpret_cast<float*>(p); }

float2* EBh(pic_ctx* ctx) { return f2(ctx->EBh); }
float2* Jh(pic_ctx* ctx) { return f2(ctx->Jh); }
float2* Gs(pic_ctx* ctx) { return f2(ctx->G); }
float2* rhoh(pic_ctx* ctx, int k) { return f2(ctx->rhoh[0]) + k * ctx->nmode; }
float* nodal(pic_ctx* ctx) { return f1(ctx->nodal); }
float* Jn(pic_ctx* ctx) { return f1(ctx->Jn); }

pic_status load_fields32(pic_ctx* ctx, const float* const E[3], const float* const B[3]) {
  CRP6<float> in;
  CP6<float2> g, eb;
  for (int c = 0; c < 3; ++c) {
    in.p[c] = E[c];
    in.p[3 + c] = B[c];
  }
  for (int c = 0; c < 6; ++c) {
    g.p[c] = Gs(ctx) + c * ctx->nmode;
    eb.p[c] = EBh(ctx) + c * ctx->nmode;
  }
  {
    StageScope t(ctx, STAGE_FFT, 3);
    PIC_TRY32(fft_r2c<float>(ctx, in, g, 6));
  }
  StageScope t(ctx, STAGE_OTHER, 1);
  return psatd_phase32(ctx, g, eb, kKindEB, 6, -1, 1.0);
}

pic_status store_yee32(pic_ctx* ctx, const float2* src, const int* kinds, int ncomp, float* const* out) {
  CP6<float2> s, g;
  RP6<float> o;
  for (int c = 0; c < ncomp; ++c) {
    s.p[c] = const_cast<float2*>(src) + c * ctx->nmode;
    g.p[c] = Gs(ctx) + c * ctx->nmode;
    o.p[c] = out[c];
  }
  {
    StageScope t(ctx, STAGE_OTHER, 1);
    PIC_TRY32(psatd_phase32(ctx, s, g, kinds, ncomp, +1, 1.0 / (double)ctx->ncell));
  }
  StageScope t(ctx, STAGE_FFT, 3);
  return fft_c2r<float>(ctx, g, o, ncomp);
}

pic_status g_to_nodal32(pic_ctx* ctx) {
  CP6<float2> g;
  RP6<float> o;
  for (int c = 0; c < 6; ++c) {
    g.p[c] = Gs(ctx) + c * ctx->nmode;
    o.p[c] = nodal(ctx) + c * ctx->ncell;
  }
  StageScope t(ctx, STAGE_FFT, 3);
  return fft_c2r<float>(ctx, g, o, 6);
}

}  // namespace

extern "C" {

pic_status pic_deposit_rho32(pic_ctx* ctx, const pic_species32* sp, int n_species, float* rho) {
  PIC_NEED_FP32(ctx);
  if (!rho) return pic_set_error(ctx, PIC_ERR_ARG, "rho is null");
  PIC_TRY32(check_species32(ctx, sp, n_species));
  PIC_CUDA_TRY(ctx, cudaMemsetAsync(rho, 0, ctx->ncell * sizeof(float), ctx->stream));
  for (int s = 0; s < n_species; ++s) PIC_TRY32(particles_deposit_rho32(ctx, &sp[s], rho));
  return PIC_OK;
}

pic_status pic_push_deposit32(pic_ctx* ctx, const float* const En[3], const float* const Bn[3],
                              const pic_species32* sp, int n_species, float* const J_nodal[3], float* rho_nodal) {
  PIC_NEED_FP32(ctx);
  if (!nonnull(En, 3) || !nonnull(Bn, 3) || !nonnull(J_nodal, 3) || !rho_nodal)
    return pic_set_error(ctx, PIC_ERR_ARG, "null field pointer");
  PIC_TRY32(check_species32(ctx, sp, n_species));
  for (int c = 0; c < 3; ++c)
    PIC_CUDA_TRY(ctx, cudaMemsetAsync(J_nodal[c], 0, ctx->ncell * sizeof(float), ctx->stream));
  PIC_CUDA_TRY(ctx, cudaMemsetAsync(rho_nodal, 0, ctx->ncell * sizeof(float), ctx->stream));
  for (int s = 0; s < n_species; ++s) PIC_TRY32(particles_push32(ctx, En, Bn, &sp[s], J_nodal, rho_nodal));
  return PIC_OK;
}

pic_status pic_bin32(pic_ctx* ctx, const pic_species32* sp, int64_t* offsets) {
  PIC_NEED_FP32(ctx);
  PIC_TRY32(check_species32(ctx, sp, 1));
  return particles_bin32(ctx, sp, offsets);
}

pic_status pic_fft_forward32(pic_ctx* ctx, const float* const real[], float* const spec[], int ncomp) {
  PIC_NEED_FP32(ctx);
  if (ncomp < 1 || ncomp > 6 || !nonnull(real, ncomp) || !nonnull(spec, ncomp))
    return pic_set_error(ctx, PIC_ERR_ARG, "fft arguments");
  PIC_NEED_ALIGNED(ctx, real, ncomp, 8);
  PIC_NEED_ALIGNED(ctx, spec, ncomp, 8);
  CRP6<float> in;
  CP6<float2> o;
  for (int c = 0; c < ncomp; ++c) {
    in.p[c] = real[c];
    o.p[c] = reinterpret_cast<float2*>(spec[c]);
  }
  return fft_r2c<float>(ctx, in, o, ncomp);
}

pic_status pic_fft_inverse32(pic_ctx* ctx, float* const spec[], float* const real[], int ncomp) {
  PIC_NEED_FP32(ctx);
  if (ncomp < 1 || ncomp > 6 || !nonnull(real, ncomp) || !nonnull(spec, ncomp))
    return pic_set_error(ctx, PIC_ERR_ARG, "fft arguments");
  PIC_NEED_ALIGNED(ctx, real, ncomp, 8);
  PIC_NEED_ALIGNED(ctx, spec, ncomp, 8);
  CP6<float2> in;
  RP6<float> o;
  for (int c = 0; c < ncomp; ++c) {
    in.p[c] = reinterpret_cast<float2*>(spec[c]);
    o.p[c] = real[c];
  }
  return fft_c2r<float>(ctx, in, o, ncomp);
}

pic_status pic_field_energy32(pic_ctx* ctx, const float* const E[3], const float* const B[3],
                              const int64_t box_lo[3], const int64_t box_hi[3], double* out) {
  PIC_NEED_FP32(ctx);
  if (!nonnull(E, 3) || !nonnull(B, 3) || !out) return pic_set_error(ctx, PIC_ERR_ARG, "null argument");
  int64_t lo[3] = {0, 0, 0}, hi[3] = {ctx->N[0], ctx->N[1], ctx->N[2]};
  if (box_lo && box_hi)
    for (int a = 0; a < 3; ++a) {
      if (box_lo[a] < 0 || box_hi[a] > ctx->N[a] || box_lo[a] > box_hi[a])
        return pic_set_error(ctx, PIC_ERR_ARG, "box out of range");
      lo[a] = box_lo[a];
      hi[a] = box_hi[a];
    }
  return diag_energy32(ctx, E, B, lo, hi, out);
}

pic_status pic_total_charge32(pic_ctx* ctx, const float* rho, double* out) {
  PIC_NEED_FP32(ctx);
  if (!rho || !out) return pic_set_error(ctx, PIC_ERR_ARG, "null argument");
  PIC_TRY32(diag_sum32(ctx, rho, out));
  *out *= ctx->dx[0] * ctx->dx[1] * ctx->dx[2];
  return PIC_OK;
}

pic_status pic_step32(pic_ctx* ctx, float* const E[3], float* const B[3], float* const J[3], float* rho,
                      const pic_species32* sp, int n_species, int nsteps) {
  PIC_NEED_FP32(ctx);
  if (!nonnull(E, 3) || !nonnull(B, 3) || (J && !nonnull(J, 3)) || !rho)
    return pic_set_error(ctx, PIC_ERR_ARG, "null field pointer");
  if (nsteps < 0) return pic_set_error(ctx, PIC_ERR_ARG, "nsteps < 0");
  {
    const void* ptrs[10] = {E[0], E[1], E[2], B[0], B[1], B[2], J ? J[0] : nullptr, J ? J[1] : nullptr,
                            J ? J[2] : nullptr, rho};
    PIC_NEED_ALIGNED(ctx, ptrs, 10, 8);
  }
  PIC_TRY32(check_species32(ctx, sp, n_species));
  if (nsteps == 0) return PIC_OK;
  const int64_t nm = ctx->nmode, nc = ctx->ncell;
  const float* cE[3] = {E[0], E[1], E[2]};
  const float* cB[3] = {B[0], B[1], B[2]};
  // FDTD cycle: the caller's Yee E, B are the state, advanced in place; no spectra.  Its Yee J is a
  // work array of the update: without the caller's, the spectral scratch.
  const bool fd = ctx->cycle == PIC_CYCLE_HYBRID_FDTD;
  float* Jw[3] = {f1(reinterpret_cast<double*>(ctx->G)), f1(reinterpret_cast<double*>(ctx->G)) + nc,
                  f1(reinterpret_cast<double*>(ctx->G)) + 2 * nc};
  float* const* Jy = J ? J : Jw;
  const float* yee[6] = {E[0], E[1], E[2], B[0], B[1], B[2]};
  float* nodal6[6];
  for (int c = 0; c < 6; ++c) nodal6[c] = nodal(ctx) + c * nc;
  const bool stag = ctx->cycle == PIC_CYCLE_STAGGERED;
  const bool tiled = ctx->sort_interval > 0 && tiled_push_fits(ctx) && !stag;
  int64_t total = 0;
  for (int q = 0; q < n_species; ++q) total += sp[q].n;
  if (tiled) {
    // device scratch of the binning (allocated once; no allocation happens inside the steps)
    if (!ctx->bin_gate) {
      PIC_CUDA_TRY(ctx, cudaMalloc(&ctx->bin_gate, sizeof(int)));
      PIC_CUDA_TRY(ctx, cudaMalloc(&ctx->bin_outside, sizeof(unsigned long long)));
      PIC_CUDA_TRY(ctx, cudaMemsetAsync(ctx->bin_outside, 0, sizeof(unsigned long long), ctx->stream));
      // drift-following tile frames: every species starts unshifted and at rest
      PIC_CUDA_TRY(ctx, cudaMalloc(&ctx->frame, 8 * PIC_MAX_BINNED_SPECIES * sizeof(int)));
      PIC_CUDA_TRY(ctx, cudaMalloc(&ctx->dhist, 10 * PIC_MAX_BINNED_SPECIES * sizeof(unsigned long long)));
      PIC_CUDA_TRY(ctx, cudaMemsetAsync(ctx->frame, 0, 8 * PIC_MAX_BINNED_SPECIES * sizeof(int), ctx->stream));
      PIC_CUDA_TRY(ctx, cudaMemsetAsync(ctx->dhist, 0, 10 * PIC_MAX_BINNED_SPECIES * sizeof(unsigned long long),
                                        ctx->stream));
    }
    for (int q = 0; q < n_species && q < PIC_MAX_BINNED_SPECIES; ++q) {
      if (!ctx->sp_off[q]) PIC_CUDA_TRY(ctx, cudaMalloc(&ctx->sp_off[q], (ctx->n_tiles + 1) * sizeof(int64_t)));
      if (!ctx->sp_chunk[q] || ctx->sp_chunk_n[q] < sp[q].n) {
        if (ctx->sp_chunk[q]) PIC_CUDA_TRY(ctx, cudaFree(ctx->sp_chunk[q]));
        ctx->sp_chunk[q] = nullptr;
        PIC_CUDA_TRY(ctx, cudaMalloc(&ctx->sp_chunk[q], tile_chunk_words(ctx, sp[q].n) * sizeof(uint32_t)));
        ctx->sp_chunk_n[q] = sp[q].n;
      }
      ctx->sp_off_n[q] = sp[q].n;
    }
  }
  // The first step's (forced) binning of species 0 reads the particles only: it runs on the
  // context's second stream, concurrently with the entry transforms of the fields on this one,
  // and the first push waits for it (fork / join by events, also valid inside graph capture).
  const bool early_bin = tiled && n_species > 0;
  if (early_bin) {
    PIC_CUDA_TRY(ctx, cudaEventRecord(ctx->ev_fork, ctx->stream));
    PIC_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->aux, ctx->ev_fork, 0));
    cudaStream_t main_stream = ctx->stream;
    ctx->stream = ctx->aux;
    pic_status st = PIC_OK;
    {
      StageScope t(ctx, STAGE_BIN, 1);
      st = particles_bin32_decide(ctx, total, 1);
    }
    if (st == PIC_OK) {
      StageScope t(ctx, STAGE_BIN, bin32_launches(ctx, sp[0].n, true, false));
      st = particles_bin32(ctx, &sp[0], ctx->sp_off[0], ctx->bin_gate, ctx->sp_chunk[0], false, ctx->frame);
    }
    ctx->stream = main_stream;
    if (st != PIC_OK) return st;
    PIC_CUDA_TRY(ctx, cudaEventRecord(ctx->ev_join, ctx->aux));
  }
  int cur = 0;
  if (!fd) {
    PIC_TRY32(load_fields32(ctx, cE, cB));
    CRP6<float> rin;
    CP6<float2> rout;
    rin.p[0] = rho;
    rout.p[0] = rhoh(ctx, cur);
    StageScope t(ctx, STAGE_FFT, 3);
    PIC_TRY32(fft_r2c<float>(ctx, rin, rout, 1));
  }
  if (fd) {
    // E^n, B^n -> nodes in real space (work arrays: the nodal J buffer, free until the deposit)
    StageScope t(ctx, STAGE_OTHER, 9);
    PIC_TRY32(center_to_nodal_t<float>(ctx, yee, nodal6, Jn(ctx), Jn(ctx) + nc));
  } else if (stag) {
    // staggered comparison cycle: the first gather reads the caller's Yee E, B as they are
    const float* src[6] = {E[0], E[1], E[2], B[0], B[1], B[2]};
    for (int c = 0; c < 6; ++c)
      PIC_CUDA_TRY(ctx, cudaMemcpyAsync(nodal(ctx) + c * nc, src[c], nc * sizeof(float), cudaMemcpyDeviceToDevice,
                                        ctx->stream));
  } else {
    {
      StageScope t(ctx, STAGE_OTHER, 1);
      PIC_TRY32(psatd_to_nodal32(ctx, EBh(ctx), Gs(ctx), 1.0 / (double)nc));
    }
    PIC_TRY32(g_to_nodal32(ctx));
  }
  float* nd = nodal(ctx);
  const float* En[3] = {nd, nd + nc, nd + 2 * nc};
  const float* Bn[3] = {nd + 3 * nc, nd + 4 * nc, nd + 5 * nc};
  float* jn = Jn(ctx);
  float* Jnp[3] = {jn, jn + nc, jn + 2 * nc};
  int since_forced = 0;
  for (int s = 0; s < nsteps; ++s) {
    const bool last = s == nsteps - 1;
    // Binning: the tiled push needs each species' tile ranges.  The first step of a call and
    // every sort_interval-th step re-bin unconditionally; in between, the device re-bins only
    // when the previous push moved more than 2 % of the particles out of their tile (they would
    // gather from global memory in the next push).
    if (tiled) {
      const int force = (s == 0 || since_forced >= ctx->sort_interval) ? 1 : 0;
      since_forced = force ? 1 : since_forced + 1;
      if (!(s == 0 && early_bin)) {  // step 0: decided on the second stream
        StageScope t(ctx, STAGE_BIN, 1);
        PIC_TRY32(particles_bin32_decide(ctx, total, force));
      }
    }
    PIC_CUDA_TRY(ctx, cudaMemsetAsync(jn, 0, 3 * nc * sizeof(float), ctx->stream));
    PIC_CUDA_TRY(ctx, cudaMemsetAsync(rho, 0, nc * sizeof(float), ctx->stream));
    for (int q = 0; q < n_species; ++q) {
      if (tiled && q < PIC_MAX_BINNED_SPECIES) {
        // the binning leaves the sorted species in the shared scratch and the push copies it back
        // (so each species is binned right before its own push)
        if (s == 0 && q == 0 && early_bin) {
          PIC_CUDA_TRY(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0));  // binned on the second stream
        } else {
          StageScope t(ctx, STAGE_BIN, bin32_launches(ctx, sp[q].n, true, false));
          PIC_TRY32(particles_bin32(ctx, &sp[q], ctx->sp_off[q], ctx->bin_gate, ctx->sp_chunk[q], false,
                                    ctx->frame + 8 * q));
        }
        // on a grid moving along z two launches: the instantiation for the species' frame velocity
        // works, its twin returns
        StageScope t(ctx, STAGE_PUSH, sp[q].n > 0 ? (ctx->vg[2] != 0.0 ? 2 : 1) : 0);
        PIC_TRY32(particles_push32_tiled(ctx, En, Bn, &sp[q], Jnp, rho, ctx->sp_off[q], ctx->sp_chunk[q],
                                         bin32_two_level(ctx) ? nullptr : bin32_scatter_gate(ctx),
                                         ctx->frame + 8 * q, ctx->dhist + 10 * q));
      } else {
        StageScope t(ctx, STAGE_PUSH, sp[q].n > 0 ? 1 : 0);
        PIC_TRY32(particles_push32(ctx, En, Bn, &sp[q], Jnp, rho));
      }
    }
    if (tiled) {
      // the tile frames follow the species' drift (binning stays off while they keep their tiles)
      StageScope t(ctx, STAGE_BIN, 1);
      PIC_TRY32(particles_frames_advance(ctx, sp, n_species));
    }
    if (fd) {
      // J^{n+1/2}: optional smoothing, nodes -> Yee (work arrays: the nodal E, B, free after the
      // push), leapfrog of E, B, then E^{n+1}, B^{n+1} -> nodes for the next gather
      {
        StageScope t(ctx, STAGE_OTHER, 3 + 9 * ctx->filter_passes);
        for (int c = 0; c < 3 && ctx->filter_passes > 0; ++c)
          PIC_TRY32(bilinear_filter_t<float>(ctx, Jnp[c], ctx->filter_passes, nodal(ctx), nodal(ctx) + nc));
        const float* cJn[3] = {Jnp[0], Jnp[1], Jnp[2]};
        PIC_TRY32(center_to_yee_t<float>(ctx, cJn, Jy, nodal(ctx), nodal(ctx) + nc));
      }
      const float* cJ[3] = {Jy[0], Jy[1], Jy[2]};
      PIC_TRY32(fdtd_update32(ctx, E, B, cJ));
      if (!last) {
        StageScope t(ctx, STAGE_OTHER, 9);
        PIC_TRY32(center_to_nodal_t<float>(ctx, yee, nodal6, Jn(ctx), Jn(ctx) + nc));
      }
      ++ctx->steps_done;
      continue;
    }
    CRP6<float> in;
    CP6<float2> out;
    for (int c = 0; c < 3; ++c) {
      in.p[c] = Jnp[c];
      out.p[c] = Jh(ctx) + c * nm;
    }
    in.p[3] = rho;
    out.p[3] = rhoh(ctx, 1 - cur);
    {
      StageScope t(ctx, STAGE_FFT, 3);
      PIC_TRY32(fft_r2c<float>(ctx, in, out, 4));
    }
    if (stag) {
      // J was deposited at its Yee positions: plain DFT -> paper convention, in place
      CP6<float2> jh;
      for (int c = 0; c < 3; ++c) jh.p[c] = Jh(ctx) + c * nm;
      StageScope t(ctx, STAGE_OTHER, 1);
      PIC_TRY32(psatd_phase32(ctx, jh, jh, kKindJ, 3, -1, 1.0));
    }
    {
      // hybrid: J nodal (centered in the update), G = nodal E, B; staggered: J and G on the Yee grid
      StageScope t(ctx, STAGE_UPDATE, 1);
      PIC_TRY32(psatd_update32(ctx, EBh(ctx), Jh(ctx), rhoh(ctx, cur), rhoh(ctx, 1 - cur), Gs(ctx), stag ? 1 : 0,
                               stag ? 1 : 0, (last && J) ? 1 : 0, 1));
    }
    cur = 1 - cur;
    if (!last) PIC_TRY32(g_to_nodal32(ctx));
    ++ctx->steps_done;
  }
  if (fd) return PIC_OK;
  float* outs[6] = {E[0], E[1], E[2], B[0], B[1], B[2]};
  PIC_TRY32(store_yee32(ctx, EBh(ctx), kKindEB, 6, outs));
  if (!J) return PIC_OK;
  float* jouts[3] = {J[0], J[1], J[2]};
  return store_yee32(ctx, Jh(ctx), kKindJ, 3, jouts);
}

}  // extern "C"
