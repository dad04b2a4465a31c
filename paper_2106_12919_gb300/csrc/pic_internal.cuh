// Internal declarations of libpic (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstring>

#include "pic.h"

#define PIC_MAX_CENTER_M 16  // centering order 2m <= 32
#define PIC_MAX_BINNED_SPECIES 8  // species that keep per-tile ranges between steps (FP32 form)

// ---------------------------------------------------------------------------
// complex helpers (double2 / float2 as (re, im))
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ double2 cmake(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ double2 cmuli(double2 a) { return make_double2(-a.y, a.x); }  // i * a
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 cmuli(float2 a) { return make_float2(-a.y, a.x); }

// Scalar / complex type pair of a precision: Real<double>::C = double2, Real<float>::C = float2.
template <class T> struct Cplx;
template <> struct Cplx<double> { using type = double2; };
template <> struct Cplx<float> { using type = float2; };
__host__ __device__ __forceinline__ double2 to_c(double2 v, double2*) { return v; }
__host__ __device__ __forceinline__ float2 to_c(double2 v, float2*) { return make_float2((float)v.x, (float)v.y); }
__host__ __device__ __forceinline__ float2 to_c(float2 v, float2*) { return v; }
template <class C> __host__ __device__ __forceinline__ C cast_c(double2 v) { return to_c(v, (C*)nullptr); }
template <class C> __host__ __device__ __forceinline__ C czero() { C z; z.x = 0; z.y = 0; return z; }

// Index of a coefficient table inside pic_ctx::coef.
enum CoefIdx {
  COEF_TC = 0, COEF_TS, COEF_X1, COEF_X2, COEF_TX3, COEF_X4,
  COEF_PSI1, COEF_PSI2, COEF_Y1, COEF_Y2, COEF_Y3, COEF_Y4, COEF_COUNT
};

// Finite-order centering weights alpha^s_{m,n}/2 of one axis (Sec. 3).
struct CenterWeights {
  int m;
  double w[PIC_MAX_CENTER_M];
};

// Per-stage device timing (CUDA events on the context stream) and launch counts.
enum TimerStage { STAGE_PUSH = 0, STAGE_FFT, STAGE_UPDATE, STAGE_BIN, STAGE_OTHER, STAGE_COUNT };
struct Timers {
  int on;
  int pool_size;
  int used;
  cudaEvent_t* pool;   // pairs (start, stop)
  int* stage;          // stage of each pair
  int64_t launches[STAGE_COUNT];
};

struct pic_ctx {
  // configuration
  int64_t N[3];
  double dx[3];
  double dt;
  int shape_order;
  int corder[3];
  int variant;
  double vg[3];
  int sorder[3];
  double c, eps0;
  int tile[3];
  int sort_interval;
  int precision;
  int filter_passes;  // bilinear smoothing passes of the deposits (0 = off)
  int pusher;         // pic_pusher
  int cycle;          // pic_cycle
  int nsm;  // streaming multiprocessors of the device (persistent kernels size their grids by it)
  cudaStream_t stream;
  cudaStream_t aux;              // second stream (FP32 step: the first binning beside the entry transforms)
  cudaEvent_t ev_fork, ev_join;  // fork / join events between stream and aux
  int64_t ncell, nzh, nmode;
  int ncoef;
  CenterWeights cw[3];
  CenterWeights fdw[3];  // FDTD cycle: staggered-difference weights alpha^s_{m,n} / ((2n - 1) dx)

  // device tables
  double* k1d;       // [3][Nmax] ks, then [3][Nmax] kc, then [3][Nmax] zeta
  double* ks[3];
  double* kc[3];
  double* zeta[3];
  double* flt1d;     // [3][Nmax] bilinear filter symbols, (cos^2(k dx / 2))^passes; NULL when off
  double* flt[3];
  float* k1d32;      // FP32 copies: [9][Nmax] as k1d, then [3][Nmax] half-cell shifts (re, im)
  float* flt32;      // FP32 copy of flt1d
  double2* twid[3];  // twiddles exp(-2 pi i j / N_a), j < N_a
  float2* twid32[3]; // the same rounded to FP32
  double2* twp;      // per-pass twiddles of the transform passes (fft_tile.cuh), and in FP32
  float2* twp32;
  double2* coef;     // [ncoef][nmode]
  // Compact copy of the tables read by the step's update (NULL when v_gal has a transverse
  // component): the coefficients depend on k_x, k_y through [k_x]_s^2, [k_y]_s^2 only, so the
  // quarter ix <= Nx/2, iy <= Ny/2 of the (kx, ky) plane holds them all ([ncoef][nqx][nqy][nzh]);
  // real doubles for the standard variant (every coefficient is real there), double2 otherwise.
  double* coefq;
  // FP32 contexts: the same rounded to FP32 (float or float2), which the FP32 update reads; it
  // rounds every FP64 coefficient to FP32 at use, so the values are the same at half the traffic
  float* coefq32;
  int coefq_real;
  int64_t nqx, nqy, nq;

  // spectral state and work (paper-convention spectra)
  double2* EBh;      // [6][nmode]: E^x..E^z, B^x..B^z
  double2* rhoh[2];  // rho^n, rho^{n+1}
  double2* Jh;       // [3][nmode]
  double2* G;        // [6][nmode] scratch for inverse transforms

  // real-space work
  double* nodal;     // [6][ncell] nodal gather fields
  double* Jn;        // [3][ncell] nodal J deposit

  // binning scratch (grown on demand)
  int64_t bin_cap;
  int32_t* bin_tid;
  int64_t* bin_counts;   // [n_tiles + 1]
  int64_t* bin_cursor;   // [n_tiles]
  double* bin_tmp;       // [8][bin_cap] permuted copies
  void* scan_tmp;
  size_t scan_tmp_bytes;
  int64_t n_tiles;
  uint32_t* cell_counts;  // FP32 binning: per-cell counts -> offsets, block sums, total
  uint32_t* cell_cursor;  // FP32 binning: per-cell scatter cursors
  double* adj_work;       // reverse mode: rhobar^n, rhobar^{n+1}, 6 nodal force adjoints
  int* bin_gate;                    // FP32 form: device flag "re-bin before the next push"
  int* bin_flags;                   // FP32 binning: [0] keys out of order, [1] scatter gate (see below)
  unsigned long long* bin_outside;  // FP32 form: particles whose new cell left their tile in the last push

  int* dev_err;  // device flag: a bounded wait of a bulk copy gave up (PIC_ERR_TIMEOUT at pic_sync)
  int64_t steps_done;
  // FP32 form: per-species tile ranges of the last binning inside pic_step32
  int64_t* sp_off[PIC_MAX_BINNED_SPECIES];
  int64_t sp_off_n[PIC_MAX_BINNED_SPECIES];   // particle count they were built for, -1 = invalid
  uint32_t* sp_chunk[PIC_MAX_BINNED_SPECIES];  // per-species chunk lists of the tiled push (see below)
  int64_t sp_chunk_n[PIC_MAX_BINNED_SPECIES];  // particle count the chunk list was sized for
  // FP32 form: drift-following tile frames, device ints per binned species q at frame + 8 q:
  // [0..2] shift of the tile grid (cells, per axis), [4..6] frame velocity (cells per step);
  // dhist + 10 q: the last push's per-axis counts of cell displacements -1, 0, +1 (and the total)
  int* frame;
  unsigned long long* dhist;
  Timers timers;
  char err[256];
};

// RAII stage scope: counts `launches` kernel launches for the stage and, when timing is on,
// brackets the enclosed work with a pair of events on the context stream.
struct StageScope {
  pic_ctx* ctx;
  int pair;
  StageScope(pic_ctx* c, int stage, int launches);
  ~StageScope();
};
void timers_free(pic_ctx* ctx);

// error helpers --------------------------------------------------------------
pic_status pic_set_error(pic_ctx* ctx, pic_status st, const char* fmt, ...);
#define PIC_CUDA_TRY(ctx, call)                                                      \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return pic_set_error((ctx), PIC_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)
#define PIC_LAUNCH_CHECK(ctx)                                                        \
  do {                                                                               \
    cudaError_t e_ = cudaGetLastError();                                             \
    if (e_ != cudaSuccess)                                                           \
      return pic_set_error((ctx), PIC_ERR_CUDA, "launch at %s:%d: %s", __FILE__, __LINE__, \
                           cudaGetErrorString(e_));                                  \
  } while (0)

#define PIC_TRY(x)               \
  do {                           \
    pic_status s_ = (x);         \
    if (s_ != PIC_OK) return s_; \
  } while (0)

// True when an output array overlaps an input array or another output array, each `bytes` long
// (stencil passes read neighbours, so they cannot run in place).
inline bool arrays_overlap(const void* const* in, int nin, const void* const* out, int nout, size_t bytes) {
  auto hit = [bytes](const void* a, const void* b) {
    const char* pa = static_cast<const char*>(a);
    const char* pb = static_cast<const char*>(b);
    return pa < pb + bytes && pb < pa + bytes;
  };
  for (int o = 0; o < nout; ++o) {
    for (int i = 0; i < nin; ++i)
      if (hit(out[o], in[i])) return true;
    for (int q = o + 1; q < nout; ++q)
      if (hit(out[o], out[q])) return true;
  }
  return false;
}

// The transforms read and write real arrays as pairs of elements (one complex value), so every real
// array given to an entry point that transforms it must start on a two-element boundary (8 bytes in
// the FP32 form, 16 in the FP64 form; every cudaMalloc or torch allocation does).  True when the
// n non-null pointers are aligned to `bytes`.
inline bool arrays_aligned(const void* const* p, int n, size_t bytes) {
  for (int i = 0; i < n; ++i)
    if (p[i] && reinterpret_cast<uintptr_t>(p[i]) % bytes != 0) return false;
  return true;
}
#define PIC_NEED_ALIGNED(ctx, ptrs, n, bytes)                                                             \
  do {                                                                                                   \
    if (!arrays_aligned(reinterpret_cast<const void* const*>(ptrs), (n), (bytes)))                       \
      return pic_set_error((ctx), PIC_ERR_ARG, "an array does not start on a %d-byte boundary", (int)(bytes)); \
  } while (0)

// Component pointer bundles passed by value to kernels.
template <class T> struct RP6 { T* p[6]; };
template <class T> struct CRP6 { const T* p[6]; };
template <class C> struct CP6 { C* p[6]; };
using RPtr6 = RP6<double>;
using CRPtr6 = CRP6<double>;
using CPtr6 = CP6<double2>;

// fft.cu ---------------------------------------------------------------------
pic_status fft_setup(pic_ctx* ctx);
// Forward R2C of ncomp real arrays into spectral arrays (plain DFT, unnormalised). T = double | float.
template <class T>
pic_status fft_r2c(pic_ctx* ctx, CRP6<T> in, CP6<typename Cplx<T>::type> out, int ncomp);
// Inverse C2R (unnormalised); spectral arrays are destroyed.
template <class T>
pic_status fft_c2r(pic_ctx* ctx, CP6<typename Cplx<T>::type> in, RP6<T> out, int ncomp);

// psatd.cu -------------------------------------------------------------------
long double fornberg_alpha_s(int m, int n);  // alpha^s_{m,n} (Eq. eq_Fornberg_staggered), host
pic_status psatd_setup(pic_ctx* ctx);   // 1D tables + per-mode coefficient tables
// Spectral update of one step. Reads ctx->EBh, ctx->Jh (nodal DFT of J), rhoh[cur], rhoh[1-cur];
// writes EBh (n+1), Jh (Yee-centered, paper convention) and G = Z * (E or <E>, B or <B>) / Ncell.
pic_status psatd_update(pic_ctx* ctx, int cur);
// General form: g_mode 0 -> G = zeta (E,B) / Ncell (nodal), 1 -> G = shift^+ (E,B) / Ncell (Yee);
// j_yee: Jh already holds the Yee-centered paper-convention spectrum; write_j: store it back;
// smooth: apply the context's bilinear filter symbols to J, rho^n, rho^{n+1} (the step's deposits).
pic_status psatd_update_ex(pic_ctx* ctx, const double2* rn, const double2* rp, int g_mode, int j_yee,
                           int write_j, int smooth);
// Multiply spectral arrays (plain DFT) by the staggering phase of each component:
// sign = -1: plain DFT -> paper convention; +1: paper convention -> plain DFT (times scale).
// comp_kind[c]: 0..5 = Ex..Bz, 6..8 = Jx..Jz, 9 = rho.
pic_status psatd_phase(pic_ctx* ctx, CPtr6 in, CPtr6 out, const int* comp_kind, int ncomp, int sign,
                       double scale);
// G[c] = Z_c * src[c] * scale, src = the six E,B spectra given (paper convention) -> nodal DFT.
pic_status psatd_to_nodal(pic_ctx* ctx, const double2* EB6, double scale);
// FP32-form counterparts (FP32 spectra, FP64 tables rounded at use).
pic_status psatd_update32(pic_ctx* ctx, float2* EB, float2* J, const float2* rn, const float2* rp, float2* G,
                          int g_mode, int j_yee, int write_j, int smooth);
pic_status psatd_phase32(pic_ctx* ctx, CP6<float2> in, CP6<float2> out, const int* comp_kind, int ncomp, int sign,
                         double scale);
pic_status psatd_to_nodal32(pic_ctx* ctx, const float2* EB6, float2* G, double scale);
// Reverse mode (adjoint.cu): conjugate-transposed update on the adjoint spectra in EB (paper
// convention, in place); G[0..2] = zeta * Jbar / Ncell (nodal DFT), G[3] = rhobar^n / Ncell,
// G[4] = rhobar^{n+1} / Ncell.
pic_status psatd_adjoint_update(pic_ctx* ctx, double2* EB, double2* G);
// EB[c] += zeta_c * src[c] (c = 0..5): transpose of the E, B -> nodal centering.
pic_status psatd_add_zeta(pic_ctx* ctx, double2* EB, const double2* src);

// Vay's pusher (J.-L. Vay, Phys. Plasmas 15, 056701 (2008); the pusher of the paper's runs,
// Secs. 5.2-5.3): u^{n+1/2} - u^{n-1/2} = (q dt / m) (E + vbar x B), vbar the mean of v^{n-1/2}
// and v^{n+1/2}, v = u / gamma, solved in closed form:
//   u' = u + (q dt / m) (E + (v^{n-1/2} x B) / 2),  tau = (q dt / (2 m)) B,
//   gamma^2 = root of gamma^4 - sigma gamma^2 - (tau^2 + (u'.tau)^2 / c^2),  sigma = 1 + u'^2 / c^2 - tau^2,
//   t = tau / gamma,  u^{n+1/2} = (u' + (u'.t) t + u' x t) / (1 + t^2).
// The positive root is taken as (sigma + R)/2 for sigma >= 0 and as 2 b / (R - sigma) for
// sigma < 0 (R = sqrt(sigma^2 + 4 b), b = tau^2 + (u'.tau)^2 / c^2): equal in exact
// arithmetic, the second avoids cancellation.  k = q dt / (2 m); f = (E, B) at the particle.
template <class T>
__device__ __forceinline__ void vay_push(T& ux, T& uy, T& uz, const T* f, T k, T inv_c2) {
  const T ig0 = T(1) / sqrt(T(1) + (ux * ux + uy * uy + uz * uz) * inv_c2);
  const T vx = ux * ig0, vy = uy * ig0, vz = uz * ig0;
  const T k2 = k + k;
  const T upx = ux + k2 * f[0] + k * (vy * f[5] - vz * f[4]);
  const T upy = uy + k2 * f[1] + k * (vz * f[3] - vx * f[5]);
  const T upz = uz + k2 * f[2] + k * (vx * f[4] - vy * f[3]);
  const T tx = k * f[3], ty = k * f[4], tz = k * f[5];
  const T tau2 = tx * tx + ty * ty + tz * tz;
  const T us = upx * tx + upy * ty + upz * tz;
  const T b = tau2 + us * us * inv_c2;
  const T sigma = T(1) + (upx * upx + upy * upy + upz * upz) * inv_c2 - tau2;
  const T R = sqrt(sigma * sigma + T(4) * b);
  const T g2 = sigma >= T(0) ? T(0.5) * (sigma + R) : T(2) * b / (R - sigma);
  const T ig = T(1) / sqrt(g2);
  const T qx = tx * ig, qy = ty * ig, qz = tz * ig;
  const T sn = T(1) / (T(1) + qx * qx + qy * qy + qz * qz);
  const T ut = upx * qx + upy * qy + upz * qz;
  ux = sn * (upx + ut * qx + (upy * qz - upz * qy));
  uy = sn * (upy + ut * qy + (upz * qx - upx * qz));
  uz = sn * (upz + ut * qz + (upx * qy - upy * qx));
}

// Read access to the update's coefficient tables: the compact quarter tables when the context has
// them, else the full [ncoef][nmode] tables.
struct CoefView {
  const double* q;       // compact tables (NULL: use full)
  const float* q32;      // their FP32 copy (FP32 contexts) or NULL
  const double2* full;   // full tables
  int real;              // compact tables hold real doubles
  int64_t nqy, nq, nmode;
  int nx, ny;            // grid sizes of the two folded axes
  __device__ __forceinline__ int64_t index(uint32_t ix, uint32_t iy, uint32_t iz, int64_t nzh) const {
    const uint32_t qx = min(ix, (uint32_t)nx - ix), qy = min(iy, (uint32_t)ny - iy);
    return ((int64_t)qx * nqy + qy) * nzh + iz;
  }
  // coefficient k of mode m = (ix, iy, iz), in FP64
  __device__ __forceinline__ double2 get(int k, int64_t m, int64_t qidx) const {
    if (q == nullptr) return __ldg(full + k * nmode + m);
    if (real) return make_double2(__ldg(q + k * nq + qidx), 0.0);
    return __ldg(reinterpret_cast<const double2*>(q) + k * nq + qidx);
  }
};
inline CoefView coef_view(const pic_ctx* ctx) {
  CoefView v;
  v.q = ctx->coefq;
  v.q32 = ctx->coefq32;
  v.full = ctx->coef;
  v.real = ctx->coefq_real;
  v.nqy = ctx->nqy;
  v.nq = ctx->nq;
  v.nmode = ctx->nmode;
  v.nx = (int)ctx->N[0];
  v.ny = (int)ctx->N[1];
  return v;
}

// index of a coefficient table by name ("TC", "TS", ..., see pic_coefficient), -1 if unknown
int coef_index(const pic_ctx* ctx, const char* name);

// particles.cu ----------------------------------------------------------------
pic_status particles_push(pic_ctx* ctx, const double* const En[3], const double* const Bn[3],
                          const pic_species* sp, double* const J[3], double* rho);
pic_status particles_deposit_rho(pic_ctx* ctx, const pic_species* sp, double* rho);
pic_status particles_bin(pic_ctx* ctx, const pic_species* sp, int64_t* offsets_out);
pic_status particles_bin_capacity(pic_ctx* ctx, int64_t n);
// FP32 form (particles32.cu)
pic_status particles_push32(pic_ctx* ctx, const float* const En[3], const float* const Bn[3],
                            const pic_species32* sp, float* const J[3], float* rho);
pic_status particles_deposit_rho32(pic_ctx* ctx, const pic_species32* sp, float* rho);
// Tiled push: one CTA per chunk of at most kTileChunk particles of one tile, over the ranges
// offsets[n_tiles + 1] of the last binning; chunks holds the exclusive prefix sum of the
// tiles' chunk counts [n_tiles + 1], its scan scratch, and the tile of every chunk.  Shared-memory deposit window per chunk.  Correct for any order
// (out-of-window deposits go global).
constexpr int kTileChunk = 2048;
bool tiled_push_fits(const pic_ctx* ctx);  // deposit window of the tile fits in shared memory
size_t tile_chunk_words(const pic_ctx* ctx, int64_t n);  // chunk list size for n particles (words)
pic_status particles_push32_tiled(pic_ctx* ctx, const float* const En[3], const float* const Bn[3],
                                  const pic_species32* sp, float* const J[3], float* rho, const int64_t* offsets,
                                  const uint32_t* chunks,
                                  const int* sorted_gate = nullptr, const int* frame = nullptr,
                                  unsigned long long* dhist = nullptr);
// gate: device flag; the binning kernels do nothing while *gate == 0 (nullptr = always bin).
// chunks_out (optional, tile_chunk_words entries): chunk starts for particles_push32_tiled.
// copy_back = false leaves the sorted particles in ctx->bin_tmp (the species arrays untouched) for
// a particles_push32_tiled call with sorted_gate = bin32_scatter_gate(ctx), which reads them there
// when the binning permuted them and writes the pushed particles to the species arrays.  A species
// already in key order gets its tile ranges only (no permutation): the scatter gate stays 0.
// frame (optional): the species' drift-following tile frame (ctx->frame + 8 q); keys are taken from
// the cell shifted by -frame[0..2].
pic_status particles_bin32(pic_ctx* ctx, const pic_species32* sp, int64_t* offsets_out, const int* gate = nullptr,
                           uint32_t* chunks_out = nullptr, bool copy_back = true, const int* frame = nullptr);
// *bin_gate = (particles whose new cell left their tile in the last tiled push > 2 % of total) || force
pic_status particles_bin32_decide(pic_ctx* ctx, int64_t total_particles, int force);
// After the pushes of a step: every binned species' tile frame moves by its frame velocity, and the
// velocity becomes the cell displacement that at least 3/4 of the species' particles made in the
// push just done (else 0); the displacement counts are cleared.
pic_status particles_frames_advance(pic_ctx* ctx, const pic_species32* sp, int n_species);
// device flag: the last particles_bin32 call permuted the species (its sorted copy is in bin_tmp)
inline const int* bin32_scatter_gate(const pic_ctx* ctx) { return ctx->bin_flags + 1; }
// tiles of at most 4096 cells are binned in two levels (by tile, then by cell inside each tile in
// shared memory), which always leaves the sorted particles in the species arrays (copy_back is
// implied); larger tiles by one counting sort over every cell
bool bin32_two_level(const pic_ctx* ctx);
// kernel launches of one particles_bin32 call (for the stage launch counters)
int bin32_launches(const pic_ctx* ctx, int64_t n, bool chunks, bool copy_back);

// center.cu -------------------------------------------------------------------
pic_status center_to_nodal(pic_ctx* ctx, const double* const F[6], double* const out[6]);
pic_status center_to_yee(pic_ctx* ctx, const double* const Jn[3], double* const out[3]);
// Either precision, with explicit work arrays w0, w1 (ncell elements each).
template <class T>
pic_status center_to_nodal_t(pic_ctx* ctx, const T* const F[6], T* const out[6], T* w0, T* w1);
template <class T>
pic_status center_to_yee_t(pic_ctx* ctx, const T* const Jn[3], T* const out[3], T* w0, T* w1);
// `passes` passes of the bilinear (1/4, 1/2, 1/4) filter along x, y, z of f in place (Sec. 2).
template <class T>
pic_status bilinear_filter_t(pic_ctx* ctx, T* f, int passes, T* w0, T* w1);

// fdtd.cu ---------------------------------------------------------------------
// Weights of the FDTD cycle's differences and its Courant check (host only, no device work).
pic_status fdtd_setup(pic_ctx* ctx);
// Leapfrog step of the Yee fields with split B, in place (see fdtd.cu).
pic_status fdtd_update(pic_ctx* ctx, double* const E[3], double* const B[3], const double* const J[3]);
pic_status fdtd_update32(pic_ctx* ctx, float* const E[3], float* const B[3], const float* const J[3]);
// nsteps of the hybrid FDTD cycle (FP64).
pic_status fdtd_step(pic_ctx* ctx, double* const E[3], double* const B[3], double* const J[3], double* rho,
                     const pic_species* sp, int n_species, int nsteps);

// diag.cu ---------------------------------------------------------------------
pic_status diag_energy(pic_ctx* ctx, const double* const E[3], const double* const B[3],
                       const int64_t lo[3], const int64_t hi[3], double* out);
pic_status diag_sum(pic_ctx* ctx, const double* a, double* out);
pic_status diag_energy32(pic_ctx* ctx, const float* const E[3], const float* const B[3],
                         const int64_t lo[3], const int64_t hi[3], double* out);
pic_status diag_sum32(pic_ctx* ctx, const float* a, double* out);

// Exact-reduction sin/cos of pi * p / q for integers (host), used to build tables.
void sincospi_frac(int64_t p, int64_t q, double* s, double* c);
