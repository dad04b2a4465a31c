// C ABI of libpic: context lifetime, argument validation and the orchestration
// of the hybrid PIC step (Sec. 2) on one stream.
#include "pic_internal.cuh"

#include <cstdarg>
#include <cstdlib>
#include <new>

int coef_index(const pic_ctx* ctx, const char* name) {
  static const char* names[COEF_COUNT] = {"TC", "TS", "X1", "X2", "TX3", "X4",
                                          "Psi1", "Psi2", "Y1", "Y2", "Y3", "Y4"};
  for (int k = 0; k < ctx->ncoef; ++k)
    if (strcmp(names[k], name) == 0) return k;
  return -1;
}

pic_status pic_set_error(pic_ctx* ctx, pic_status st, const char* fmt, ...) {
  if (ctx) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
    va_end(ap);
  }
  return st;
}

namespace {

bool pow2_in(int64_t n, int64_t lo, int64_t hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }

template <class T>
pic_status dalloc(pic_ctx* ctx, T** p, size_t count, const char* what) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return pic_set_error(ctx, PIC_ERR_NOMEM, "cudaMalloc %s (%zu bytes): %s", what, count * sizeof(T),
                         cudaGetErrorString(e));
  }
  return PIC_OK;
}

pic_status check_species(pic_ctx* ctx, const pic_species* sp, int n_species) {
  if (n_species < 0 || (n_species > 0 && sp == nullptr)) return pic_set_error(ctx, PIC_ERR_ARG, "species array");
  for (int s = 0; s < n_species; ++s) {
    const pic_species& p = sp[s];
    if (p.n < 0) return pic_set_error(ctx, PIC_ERR_ARG, "species %d: negative count", s);
    if (p.n > 0 && (!p.x || !p.y || !p.z || !p.ux || !p.uy || !p.uz || !p.w))
      return pic_set_error(ctx, PIC_ERR_ARG, "species %d: null array", s);
    if (!(p.m > 0.0)) return pic_set_error(ctx, PIC_ERR_ARG, "species %d: mass must be > 0", s);
    if (p.n > ((int64_t)1 << 31) - 1)
      return pic_set_error(ctx, PIC_ERR_CAPACITY, "species %d: more than 2^31-1 particles", s);
  }
  return PIC_OK;
}

template <class P>
bool all_nonnull(P const* a, int n) {
  if (!a) return false;
  for (int i = 0; i < n; ++i)
    if (!a[i]) return false;
  return true;
}

const int kKindEB[6] = {0, 1, 2, 3, 4, 5};
const int kKindJ[3] = {6, 7, 8};

// Yee E, B (real) -> ctx->EBh (paper-convention spectra), via G as scratch.
pic_status load_fields(pic_ctx* ctx, const double* const E[3], const double* const B[3]) {
  CRPtr6 in;
  CPtr6 g, eb;
  for (int c = 0; c < 3; ++c) {
    in.p[c] = E[c];
    in.p[3 + c] = B[c];
  }
  for (int c = 0; c < 6; ++c) {
    g.p[c] = ctx->G + c * ctx->nmode;
    eb.p[c] = ctx->EBh + c * ctx->nmode;
  }
  {
    StageScope t(ctx, STAGE_FFT, 3);
    PIC_TRY(fft_r2c(ctx, in, g, 6));
  }
  StageScope t(ctx, STAGE_OTHER, 1);
  return psatd_phase(ctx, g, eb, kKindEB, 6, -1, 1.0);
}

// spectra (paper convention) -> Yee real arrays, through G.
pic_status store_yee(pic_ctx* ctx, const double2* src, const int* kinds, int ncomp, double* const* out) {
  CPtr6 s, g;
  RPtr6 o;
  for (int c = 0; c < ncomp; ++c) {
    s.p[c] = const_cast<double2*>(src) + c * ctx->nmode;
    g.p[c] = ctx->G + c * ctx->nmode;
    o.p[c] = out[c];
  }
  {
    StageScope t(ctx, STAGE_OTHER, 1);
    PIC_TRY(psatd_phase(ctx, s, g, kinds, ncomp, +1, 1.0 / (double)ctx->ncell));
  }
  StageScope t(ctx, STAGE_FFT, 3);
  return fft_c2r(ctx, g, o, ncomp);
}

// G (nodal spectra, already scaled) -> ctx->nodal real arrays.
pic_status g_to_nodal(pic_ctx* ctx) {
  CPtr6 g;
  RPtr6 o;
  for (int c = 0; c < 6; ++c) {
    g.p[c] = ctx->G + c * ctx->nmode;
    o.p[c] = ctx->nodal + c * ctx->ncell;
  }
  StageScope t(ctx, STAGE_FFT, 3);
  return fft_c2r(ctx, g, o, 6);
}

}  // namespace

extern "C" {

void pic_ext_default(pic_ext* e) {
  if (!e) return;
  memset(e, 0, sizeof(*e));
  e->struct_size = sizeof(pic_ext);
  e->precision = PIC_FP64;
  e->c = 1.0;
  e->eps0 = 1.0;
  e->tile[0] = e->tile[1] = e->tile[2] = 8;
  e->sort_interval = 20;
  e->cuda_stream = nullptr;
}

void pic_destroy(pic_ctx* ctx) {
  if (!ctx) return;
  void* ptrs[] = {ctx->k1d, ctx->twid[0], ctx->twid[1], ctx->twid[2], ctx->twid32[0], ctx->twid32[1], ctx->twid32[2], ctx->twp, ctx->twp32, ctx->coef, ctx->EBh,
                  ctx->rhoh[0], ctx->Jh, ctx->G, ctx->nodal, ctx->Jn, ctx->bin_tid, ctx->bin_counts,
                  ctx->bin_cursor, ctx->bin_tmp, ctx->cell_counts, ctx->cell_cursor, ctx->adj_work, ctx->bin_gate,
                  ctx->bin_outside, ctx->flt1d, ctx->bin_flags, ctx->k1d32, ctx->flt32, ctx->coefq,
                  ctx->coefq32, ctx->frame, ctx->dhist, ctx->dev_err};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (int q = 0; q < PIC_MAX_BINNED_SPECIES; ++q) {
    if (ctx->sp_off[q]) cudaFree(ctx->sp_off[q]);
    if (ctx->sp_chunk[q]) cudaFree(ctx->sp_chunk[q]);
  }
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->aux) cudaStreamDestroy(ctx->aux);
  timers_free(ctx);
  delete ctx;
}

const char* pic_last_error(const pic_ctx* ctx) { return ctx ? ctx->err : "null context"; }

pic_status pic_init(pic_ctx** out, const int64_t grid[3], const double dx[3], double dt, int shape_order,
                    const int32_t centering_order[3], int psatd_variant, const double v_gal[3],
                    const pic_ext* ext) {
  if (!out) return PIC_ERR_ARG;
  *out = nullptr;
  pic_ctx* ctx = new (std::nothrow) pic_ctx();
  if (!ctx) return PIC_ERR_NOMEM;
  pic_ext e;
  pic_ext_default(&e);
  if (ext) {
    if (ext->struct_size != sizeof(pic_ext)) {
      pic_destroy(ctx);
      return PIC_ERR_ARG;
    }
    e = *ext;
  }
  pic_status st = PIC_OK;
  auto fail = [&](pic_status s, const char* msg) {
    fprintf(stderr, "pic_init: %s\n", msg);
    pic_destroy(ctx);
    return s;
  };
  if (!grid || !dx || !centering_order) return fail(PIC_ERR_ARG, "null argument");
  for (int a = 0; a < 3; ++a) {
    if (!pow2_in(grid[a], a == 2 ? 16 : 8, 1024)) return fail(PIC_ERR_UNSUPPORTED, "grid sizes must be powers of two in [8,1024] (Nz >= 16)");
    if (!(dx[a] > 0.0)) return fail(PIC_ERR_ARG, "dx must be > 0");
    const int co = centering_order[a];
    if (co < 2 || co % 2 || co / 2 > PIC_MAX_CENTER_M || co > grid[a]) return fail(PIC_ERR_ARG, "centering order must be even, 2..32 and <= N");
    const int so = e.spectral_order[a];
    if (so < 0 || so % 2 || so > grid[a]) return fail(PIC_ERR_ARG, "spectral order must be 0 or even and <= N");
    if (!pow2_in(e.tile[a], 1, grid[a])) return fail(PIC_ERR_ARG, "tile edges must be powers of two dividing the grid");
  }
  if (!(dt > 0.0)) return fail(PIC_ERR_ARG, "dt must be > 0");
  if (shape_order < 1 || shape_order > 3) return fail(PIC_ERR_ARG, "shape order must be 1, 2 or 3");
  if (psatd_variant < 0 || psatd_variant > 2) return fail(PIC_ERR_ARG, "unknown PSATD variant");
  if (e.precision != PIC_FP64 && e.precision != PIC_FP32) return fail(PIC_ERR_ARG, "precision must be PIC_FP64 or PIC_FP32");
  if (!(e.c > 0.0) || !(e.eps0 > 0.0)) return fail(PIC_ERR_ARG, "c and eps0 must be > 0");
  if (e.filter_passes < 0 || e.filter_passes > 8) return fail(PIC_ERR_ARG, "filter_passes must be in [0, 8]");
  if (e.pusher != PIC_PUSHER_BORIS && e.pusher != PIC_PUSHER_VAY) return fail(PIC_ERR_ARG, "unknown pusher");
  if (e.cycle < PIC_CYCLE_HYBRID || e.cycle > PIC_CYCLE_HYBRID_FDTD) return fail(PIC_ERR_ARG, "unknown cycle");
  if (e.cycle == PIC_CYCLE_HYBRID_FDTD && psatd_variant != PIC_PSATD_STANDARD)
    return fail(PIC_ERR_UNSUPPORTED, "the FDTD cycle has the standard (non-Galilean) update only");
  if (e.cycle == PIC_CYCLE_HYBRID_FDTD)
    for (int a = 0; a < 3; ++a)
      if (e.spectral_order[a] / 2 > PIC_MAX_CENTER_M)
        return fail(PIC_ERR_ARG, "FDTD difference order must be <= 32");
  if (e.reserved) return fail(PIC_ERR_ARG, "reserved fields must be 0");
  if (psatd_variant != PIC_PSATD_STANDARD) {
    if (!v_gal) return fail(PIC_ERR_ARG, "v_gal required");
    const double v2 = v_gal[0] * v_gal[0] + v_gal[1] * v_gal[1] + v_gal[2] * v_gal[2];
    if (!(v2 < e.c * e.c)) return fail(PIC_ERR_ARG, "|v_gal| must be < c");
  }
  for (int a = 0; a < 3; ++a) {
    ctx->N[a] = grid[a];
    ctx->dx[a] = dx[a];
    ctx->corder[a] = centering_order[a];
    ctx->sorder[a] = e.spectral_order[a];
    ctx->tile[a] = e.tile[a];
    ctx->vg[a] = (psatd_variant != PIC_PSATD_STANDARD) ? v_gal[a] : 0.0;
  }
  ctx->dt = dt;
  ctx->shape_order = shape_order;
  ctx->variant = psatd_variant;
  ctx->c = e.c;
  ctx->eps0 = e.eps0;
  ctx->sort_interval = e.sort_interval;
  ctx->precision = e.precision;
  ctx->filter_passes = e.filter_passes;
  ctx->pusher = e.pusher;
  ctx->cycle = e.cycle;
  for (int q = 0; q < PIC_MAX_BINNED_SPECIES; ++q) ctx->sp_off_n[q] = -1;
  ctx->stream = reinterpret_cast<cudaStream_t>(e.cuda_stream);
  if (ctx->cycle == PIC_CYCLE_HYBRID_FDTD && (st = fdtd_setup(ctx)) != PIC_OK) {
    fprintf(stderr, "pic_init: %s\n", ctx->err);
    pic_destroy(ctx);
    return st;
  }
  ctx->ncell = grid[0] * grid[1] * grid[2];
  ctx->nzh = grid[2] / 2 + 1;
  ctx->nmode = grid[0] * grid[1] * ctx->nzh;
  ctx->n_tiles = (grid[0] / e.tile[0]) * (grid[1] / e.tile[1]) * (grid[2] / e.tile[2]);

  const size_t nm = ctx->nmode, nc = ctx->ncell;
  if ((st = dalloc(ctx, &ctx->EBh, 6 * nm, "E,B spectra")) != PIC_OK ||
      (st = dalloc(ctx, &ctx->rhoh[0], 2 * nm, "rho spectra")) != PIC_OK ||
      (st = dalloc(ctx, &ctx->Jh, 3 * nm, "J spectra")) != PIC_OK ||
      (st = dalloc(ctx, &ctx->G, 6 * nm, "scratch spectra")) != PIC_OK ||
      (st = dalloc(ctx, &ctx->nodal, 6 * nc, "nodal fields")) != PIC_OK ||
      (st = dalloc(ctx, &ctx->Jn, 3 * nc, "nodal J")) != PIC_OK) {
    fprintf(stderr, "pic_init: %s\n", ctx->err);
    pic_destroy(ctx);
    return st;
  }
  ctx->rhoh[1] = ctx->rhoh[0] + nm;
  if ((st = [&]() -> pic_status {
         PIC_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking));
         PIC_CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
         PIC_CUDA_TRY(ctx, cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
         PIC_CUDA_TRY(ctx, cudaMalloc(&ctx->dev_err, sizeof(int)));
         PIC_CUDA_TRY(ctx, cudaMemset(ctx->dev_err, 0, sizeof(int)));
         return PIC_OK;
       }()) != PIC_OK) {
    fprintf(stderr, "pic_init: %s\n", ctx->err);
    pic_destroy(ctx);
    return st;
  }
  if ((st = fft_setup(ctx)) != PIC_OK || (st = psatd_setup(ctx)) != PIC_OK) {
    fprintf(stderr, "pic_init: %s\n", ctx->err);
    pic_destroy(ctx);
    return st;
  }
  *out = ctx;
  return PIC_OK;
}

pic_status pic_sync(pic_ctx* ctx) {
  if (!ctx) return PIC_ERR_ARG;
  PIC_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  PIC_CUDA_TRY(ctx, cudaGetLastError());
  int err = 0;
  PIC_CUDA_TRY(ctx, cudaMemcpy(&err, ctx->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    PIC_CUDA_TRY(ctx, cudaMemset(ctx->dev_err, 0, sizeof(int)));
    return pic_set_error(ctx, PIC_ERR_TIMEOUT, "a bounded wait for a bulk copy gave up; the results are invalid");
  }
  return PIC_OK;
}

int64_t pic_num_tiles(const pic_ctx* ctx) { return ctx ? ctx->n_tiles : -1; }

pic_status pic_deposit_rho(pic_ctx* ctx, const pic_species* sp, int n_species, double* rho) {
  if (!ctx) return PIC_ERR_ARG;
  if (ctx->precision != PIC_FP64) return pic_set_error(ctx, PIC_ERR_ARG, "FP64 entry point on an FP32 context");
  if (!rho) return pic_set_error(ctx, PIC_ERR_ARG, "rho is null");
  PIC_TRY(check_species(ctx, sp, n_species));
  PIC_CUDA_TRY(ctx, cudaMemsetAsync(rho, 0, ctx->ncell * sizeof(double), ctx->stream));
  for (int s = 0; s < n_species; ++s) PIC_TRY(particles_deposit_rho(ctx, &sp[s], rho));
  return PIC_OK;
}

pic_status pic_push_deposit(pic_ctx* ctx, const double* const En[3], const double* const Bn[3],
                            const pic_species* sp, int n_species, double* const J_nodal[3], double* rho_nodal) {
  if (!ctx) return PIC_ERR_ARG;
  if (ctx->precision != PIC_FP64) return pic_set_error(ctx, PIC_ERR_ARG, "FP64 entry point on an FP32 context");
  if (!all_nonnull(En, 3) || !all_nonnull(Bn, 3) || !all_nonnull(J_nodal, 3) || !rho_nodal)
    return pic_set_error(ctx, PIC_ERR_ARG, "null field pointer");
  PIC_TRY(check_species(ctx, sp, n_species));
  for (int c = 0; c < 3; ++c)
    PIC_CUDA_TRY(ctx, cudaMemsetAsync(J_nodal[c], 0, ctx->ncell * sizeof(double), ctx->stream));
  PIC_CUDA_TRY(ctx, cudaMemsetAsync(rho_nodal, 0, ctx->ncell * sizeof(double), ctx->stream));
  for (int s = 0; s < n_species; ++s) PIC_TRY(particles_push(ctx, En, Bn, &sp[s], J_nodal, rho_nodal));
  return PIC_OK;
}

pic_status pic_bin(pic_ctx* ctx, const pic_species* sp, int64_t* offsets) {
  if (!ctx) return PIC_ERR_ARG;
  if (ctx->precision != PIC_FP64) return pic_set_error(ctx, PIC_ERR_ARG, "FP64 entry point on an FP32 context");
  PIC_TRY(check_species(ctx, sp, 1));
  return particles_bin(ctx, sp, offsets);
}

pic_status pic_center_to_nodal(pic_ctx* ctx, const double* const F[6], double* const out[6]) {
  if (!ctx) return PIC_ERR_ARG;
  if (ctx->precision != PIC_FP64) return pic_set_error(ctx, PIC_ERR_ARG, "FP64 entry point on an FP32 context");
  if (!all_nonnull(F, 6) || !all_nonnull(out, 6)) return pic_set_error(ctx, PIC_ERR_ARG, "null field pointer");
  if (arrays_overlap(reinterpret_cast<const void* const*>(F), 6, reinterpret_cast<const void* const*>(out), 6,
                     ctx->ncell * sizeof(double)))
    return pic_set_error(ctx, PIC_ERR_ARG, "an output array overlaps an input or another output");
  return center_to_nodal(ctx, F, out);
}

pic_status pic_center_to_yee(pic_ctx* ctx, const double* const Jn[3], double* const out[3]) {
  if (!ctx) return PIC_ERR_ARG;
  if (ctx->precision != PIC_FP64) return pic_set_error(ctx, PIC_ERR_ARG, "FP64 entry point on an FP32 context");
  if (!all_nonnull(Jn, 3) || !all_nonnull(out, 3)) return pic_set_error(ctx, PIC_ERR_ARG, "null field pointer");
  if (arrays_overlap(reinterpret_cast<const void* const*>(Jn), 3, reinterpret_cast<const void* const*>(out), 3,
                     ctx->ncell * sizeof(double)))
    return pic_set_error(ctx, PIC_ERR_ARG, "an output array overlaps an input or another output");
  return center_to_yee(ctx, Jn, out);
}

pic_status pic_fft_forward(pic_ctx* ctx, const double* const real[], double* const spec[], int ncomp) {
  if (!ctx) return PIC_ERR_ARG;
  if (ctx->precision != PIC_FP64) return pic_set_error(ctx, PIC_ERR_ARG, "FP64 entry point on an FP32 context");
  if (ncomp < 1 || ncomp > 6 || !all_nonnull(real, ncomp) || !all_nonnull(spec, ncomp))
    return pic_set_error(ctx, PIC_ERR_ARG, "fft arguments");
  PIC_NEED_ALIGNED(ctx, real, ncomp, 16);
  PIC_NEED_ALIGNED(ctx, spec, ncomp, 16);
  CRPtr6 in;
  CPtr6 o;
  for (int c = 0; c < ncomp; ++c) {
    in.p[c] = real[c];
    o.p[c] = reinterpret_cast<double2*>(spec[c]);
  }
  return fft_r2c(ctx, in, o, ncomp);
}

pic_status pic_fft_inverse(pic_ctx* ctx, double* const spec[], double* const real[], int ncomp) {
  if (!ctx) return PIC_ERR_ARG;
  if (ctx->precision != PIC_FP64) return pic_set_error(ctx, PIC_ERR_ARG, "FP64 entry point on an FP32 context");
  if (ncomp < 1 || ncomp > 6 || !all_nonnull(real, ncomp) || !all_nonnull(spec, ncomp))
    return pic_set_error(ctx, PIC_ERR_ARG, "fft arguments");
  PIC_NEED_ALIGNED(ctx, real, ncomp, 16);
  PIC_NEED_ALIGNED(ctx, spec, ncomp, 16);
  CPtr6 in;
  RPtr6 o;
  for (int c = 0; c < ncomp; ++c) {
    in.p[c] = reinterpret_cast<double2*>(spec[c]);
    o.p[c] = real[c];
  }
  return fft_c2r(ctx, in, o, ncomp);
}

pic_status pic_maxwell_step(pic_ctx* ctx, double* const E[3], double* const B[3], const double* const J[3],
                            const double* rho_n, const double* rho_np1, double* const Eavg[3],
                            double* const Bavg[3]) {
  if (!ctx) return PIC_ERR_ARG;
  if (ctx->precision != PIC_FP64) return pic_set_error(ctx, PIC_ERR_ARG, "FP64 entry point on an FP32 context");
  if (!all_nonnull(E, 3) || !all_nonnull(B, 3) || !all_nonnull(J, 3))
    return pic_set_error(ctx, PIC_ERR_ARG, "null field pointer");
  {
    const void* ptrs[11] = {E[0], E[1], E[2], B[0], B[1], B[2], J[0], J[1], J[2], rho_n, rho_np1};
    PIC_NEED_ALIGNED(ctx, ptrs, 11, 16);
    const void* avg[6] = {Eavg ? Eavg[0] : nullptr, Eavg ? Eavg[1] : nullptr, Eavg ? Eavg[2] : nullptr,
                          Bavg ? Bavg[0] : nullptr, Bavg ? Bavg[1] : nullptr, Bavg ? Bavg[2] : nullptr};
    PIC_NEED_ALIGNED(ctx, avg, 6, 16);
  }
  if (ctx->cycle == PIC_CYCLE_HYBRID_FDTD) {
    const double* cJ[3] = {J[0], J[1], J[2]};
    return fdtd_update(ctx, E, B, cJ);
  }
  if (!rho_n || !rho_np1) return pic_set_error(ctx, PIC_ERR_ARG, "null field pointer");
  const bool avg = ctx->variant == PIC_PSATD_AVERAGED_GALILEAN;
  if (avg && (!all_nonnull(Eavg, 3) || !all_nonnull(Bavg, 3)))
    return pic_set_error(ctx, PIC_ERR_ARG, "averaged variant needs Eavg, Bavg");
  const double* cE[3] = {E[0], E[1], E[2]};
  const double* cB[3] = {B[0], B[1], B[2]};
  PIC_TRY(load_fields(ctx, cE, cB));
  // J (Yee) -> Jh paper convention; rho^n, rho^{n+1} -> rhoh
  CRPtr6 in;
  CPtr6 g, jh;
  for (int c = 0; c < 3; ++c) {
    in.p[c] = J[c];
    g.p[c] = ctx->G + c * ctx->nmode;
    jh.p[c] = ctx->Jh + c * ctx->nmode;
  }
  PIC_TRY(fft_r2c(ctx, in, g, 3));
  PIC_TRY(psatd_phase(ctx, g, jh, kKindJ, 3, -1, 1.0));
  CRPtr6 rin;
  CPtr6 rout;
  rin.p[0] = rho_n;
  rin.p[1] = rho_np1;
  rout.p[0] = ctx->rhoh[0];
  rout.p[1] = ctx->rhoh[1];
  PIC_TRY(fft_r2c(ctx, rin, rout, 2));
  PIC_TRY(psatd_update_ex(ctx, ctx->rhoh[0], ctx->rhoh[1], 1, 1, 0, 0));
  if (avg) {
    RPtr6 o;
    CPtr6 gg;
    for (int c = 0; c < 3; ++c) {
      o.p[c] = Eavg[c];
      o.p[3 + c] = Bavg[c];
    }
    for (int c = 0; c < 6; ++c) gg.p[c] = ctx->G + c * ctx->nmode;
    PIC_TRY(fft_c2r(ctx, gg, o, 6));
  }
  double* outs[6] = {E[0], E[1], E[2], B[0], B[1], B[2]};
  return store_yee(ctx, ctx->EBh, kKindEB, 6, outs);
}

pic_status pic_coefficient(pic_ctx* ctx, const char* name, double* out) {
  if (!ctx) return PIC_ERR_ARG;
  if (!name || !out) return pic_set_error(ctx, PIC_ERR_ARG, "null argument");
  const int k = coef_index(ctx, name);
  if (k < 0) return pic_set_error(ctx, PIC_ERR_ARG, "unknown coefficient '%s'", name);
  PIC_CUDA_TRY(ctx, cudaMemcpyAsync(out, ctx->coef + k * ctx->nmode, ctx->nmode * sizeof(double2),
                                    cudaMemcpyDeviceToDevice, ctx->stream));
  return PIC_OK;
}

pic_status pic_field_energy(pic_ctx* ctx, const double* const E[3], const double* const B[3],
                            const int64_t box_lo[3], const int64_t box_hi[3], double* out) {
  if (!ctx) return PIC_ERR_ARG;
  if (ctx->precision != PIC_FP64) return pic_set_error(ctx, PIC_ERR_ARG, "FP64 entry point on an FP32 context");
  if (!all_nonnull(E, 3) || !all_nonnull(B, 3) || !out) return pic_set_error(ctx, PIC_ERR_ARG, "null argument");
  int64_t lo[3] = {0, 0, 0}, hi[3] = {ctx->N[0], ctx->N[1], ctx->N[2]};
  if (box_lo && box_hi)
    for (int a = 0; a < 3; ++a) {
      if (box_lo[a] < 0 || box_hi[a] > ctx->N[a] || box_lo[a] > box_hi[a])
        return pic_set_error(ctx, PIC_ERR_ARG, "box out of range");
      lo[a] = box_lo[a];
      hi[a] = box_hi[a];
    }
  return diag_energy(ctx, E, B, lo, hi, out);
}

pic_status pic_total_charge(pic_ctx* ctx, const double* rho, double* out) {
  if (!ctx) return PIC_ERR_ARG;
  if (ctx->precision != PIC_FP64) return pic_set_error(ctx, PIC_ERR_ARG, "FP64 entry point on an FP32 context");
  if (!rho || !out) return pic_set_error(ctx, PIC_ERR_ARG, "null argument");
  PIC_TRY(diag_sum(ctx, rho, out));
  *out *= ctx->dx[0] * ctx->dx[1] * ctx->dx[2];
  return PIC_OK;
}

pic_status pic_step(pic_ctx* ctx, double* const E[3], double* const B[3], double* const J[3], double* rho,
                    const pic_species* sp, int n_species, int nsteps) {
  if (!ctx) return PIC_ERR_ARG;
  if (ctx->precision != PIC_FP64) return pic_set_error(ctx, PIC_ERR_ARG, "FP64 entry point on an FP32 context");
  if (!all_nonnull(E, 3) || !all_nonnull(B, 3) || (J && !all_nonnull(J, 3)) || !rho)
    return pic_set_error(ctx, PIC_ERR_ARG, "null field pointer");
  if (nsteps < 0) return pic_set_error(ctx, PIC_ERR_ARG, "nsteps < 0");
  {
    const void* ptrs[10] = {E[0], E[1], E[2], B[0], B[1], B[2], J ? J[0] : nullptr, J ? J[1] : nullptr,
                            J ? J[2] : nullptr, rho};
    PIC_NEED_ALIGNED(ctx, ptrs, 10, 16);
  }
  PIC_TRY(check_species(ctx, sp, n_species));
  if (nsteps == 0) return PIC_OK;
  if (ctx->cycle == PIC_CYCLE_HYBRID_FDTD) {
    // the Yee J is a work array of the FDTD update: without the caller's, the spectral scratch
    double* g = reinterpret_cast<double*>(ctx->G);
    double* Jw[3] = {g, g + ctx->ncell, g + 2 * ctx->ncell};
    return fdtd_step(ctx, E, B, J ? J : Jw, rho, sp, n_species, nsteps);
  }
  const int64_t nm = ctx->nmode, nc = ctx->ncell;
  // entry: spectral E^n, B^n, rho^n; nodal gather fields
  const double* cE[3] = {E[0], E[1], E[2]};
  const double* cB[3] = {B[0], B[1], B[2]};
  PIC_TRY(load_fields(ctx, cE, cB));
  int cur = 0;
  {
    CRPtr6 rin;
    CPtr6 rout;
    rin.p[0] = rho;
    rout.p[0] = ctx->rhoh[cur];
    StageScope t(ctx, STAGE_FFT, 3);
    PIC_TRY(fft_r2c(ctx, rin, rout, 1));
  }
  const bool stag = ctx->cycle == PIC_CYCLE_STAGGERED;
  if (stag) {
    // staggered comparison cycle: the first gather reads the caller's Yee E, B as they are
    const double* src[6] = {E[0], E[1], E[2], B[0], B[1], B[2]};
    for (int c = 0; c < 6; ++c)
      PIC_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->nodal + c * nc, src[c], nc * sizeof(double), cudaMemcpyDeviceToDevice,
                                        ctx->stream));
  } else {
    {
      StageScope t(ctx, STAGE_OTHER, 1);
      PIC_TRY(psatd_to_nodal(ctx, ctx->EBh, 1.0 / (double)nc));
    }
    PIC_TRY(g_to_nodal(ctx));
  }
  const double* En[3] = {ctx->nodal, ctx->nodal + nc, ctx->nodal + 2 * nc};
  const double* Bn[3] = {ctx->nodal + 3 * nc, ctx->nodal + 4 * nc, ctx->nodal + 5 * nc};
  double* Jn[3] = {ctx->Jn, ctx->Jn + nc, ctx->Jn + 2 * nc};
  for (int s = 0; s < nsteps; ++s) {
    const bool last = s == nsteps - 1;
    if (ctx->sort_interval > 0 && ctx->steps_done % ctx->sort_interval == 0)
      for (int q = 0; q < n_species; ++q) {
        StageScope t(ctx, STAGE_BIN, sp[q].n > 0 ? 3 : 1);
        PIC_TRY(particles_bin(ctx, &sp[q], nullptr));
      }
    PIC_CUDA_TRY(ctx, cudaMemsetAsync(ctx->Jn, 0, 3 * nc * sizeof(double), ctx->stream));
    PIC_CUDA_TRY(ctx, cudaMemsetAsync(rho, 0, nc * sizeof(double), ctx->stream));
    for (int q = 0; q < n_species; ++q) {
      StageScope t(ctx, STAGE_PUSH, sp[q].n > 0 ? 1 : 0);
      PIC_TRY(particles_push(ctx, En, Bn, &sp[q], Jn, rho));
    }
    CRPtr6 in;
    CPtr6 out;
    for (int c = 0; c < 3; ++c) {
      in.p[c] = Jn[c];
      out.p[c] = ctx->Jh + c * nm;
    }
    in.p[3] = rho;
    out.p[3] = ctx->rhoh[1 - cur];
    {
      StageScope t(ctx, STAGE_FFT, 3);
      PIC_TRY(fft_r2c(ctx, in, out, 4));
    }
    if (stag) {
      // J was deposited at its Yee positions: plain DFT -> paper convention, in place
      CPtr6 jh;
      for (int c = 0; c < 3; ++c) jh.p[c] = ctx->Jh + c * nm;
      StageScope t(ctx, STAGE_OTHER, 1);
      PIC_TRY(psatd_phase(ctx, jh, jh, kKindJ, 3, -1, 1.0));
    }
    {
      // hybrid: J nodal (centered in the update), G = nodal E, B; staggered: J and G on the Yee grid
      StageScope t(ctx, STAGE_UPDATE, 1);
      PIC_TRY(psatd_update_ex(ctx, ctx->rhoh[cur], ctx->rhoh[1 - cur], stag ? 1 : 0, stag ? 1 : 0,
                              (last && J) ? 1 : 0, 1));
    }
    cur = 1 - cur;
    if (!last) PIC_TRY(g_to_nodal(ctx));
    ++ctx->steps_done;
  }
  // exit: Yee E, B and J
  double* outs[6] = {E[0], E[1], E[2], B[0], B[1], B[2]};
  PIC_TRY(store_yee(ctx, ctx->EBh, kKindEB, 6, outs));
  if (!J) return PIC_OK;
  double* jouts[3] = {J[0], J[1], J[2]};
  return store_yee(ctx, ctx->Jh, kKindJ, 3, jouts);
}

}  // extern "C"
