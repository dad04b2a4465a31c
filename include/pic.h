/*
 * libpic: hybrid nodal-staggered PSATD particle-in-cell step on one GB300.
 *
 * Method: Zoni et al., "A Hybrid Nodal-Staggered Pseudo-Spectral Electromagnetic
 * Particle-In-Cell Method with Finite-Order Centering" (arXiv 2106.12919).
 * One step follows the hybrid cycle of Sec. 2: gather E, B from a nodal grid,
 * push particles, deposit J and rho on the nodal grid, center J to the Yee grid
 * with finite-order Fornberg stencils (Sec. 3), solve Maxwell's equations on the
 * Yee grid in Fourier space with a PSATD update (Sec. 4: standard, Galilean or
 * averaged Galilean), and center E, B back to the nodal grid.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Units: SI-like with c and eps0 as parameters (mu0 = 1 / (eps0 c^2)).
 * Grid: Nx x Ny x Nz cells, periodic on every axis, each N a power of two in
 *   [8, 1024].  Node (i, j, k) is at (i dx, j dy, k dz).
 * Real-space arrays: one array per component, C order [Nx][Ny][Nz] (z fastest),
 *   element type double (PIC_FP64).  Yee positions (App. A): E^x, J^x at
 *   (i+1/2, j, k); E^y, J^y at (i, j+1/2, k); E^z, J^z at (i, j, k+1/2);
 *   B^x at (i, j+1/2, k+1/2); B^y at (i+1/2, j, k+1/2); B^z at (i+1/2, j+1/2, k);
 *   rho nodal.  "Nodal" arrays hold every component at (i, j, k).
 * Spectral arrays (only the FFT entry points expose them): complex interleaved
 *   (re, im), C order [Nx][Ny][Nz/2+1], plain DFT sum_j f_j exp(-2 pi i j.m / N)
 *   with no normalisation on the forward transform.
 * Pointers: every field and particle pointer is DEVICE memory owned by the
 *   caller, never freed or retained by the library; "host" pointers are named
 *   as such.  The transforms treat pairs of real elements as one complex value,
 *   so the field arrays given to pic_step / pic_step32, pic_maxwell_step,
 *   pic_adjoint_step and the pic_fft_* calls must start on a two-element
 *   boundary (16 bytes for double, 8 for float; every cudaMalloc or torch
 *   allocation does): PIC_ERR_ARG otherwise.  Work buffers, coefficient tables and the spectral field state
 *   belong to the context.
 * Streams: all work is enqueued on the context's stream (pic_ext.cuda_stream,
 *   default: the legacy default stream).  pic_step32 runs the first binning of a
 *   call on a second stream that the context owns, forked from and joined back
 *   into the context's stream by events inside the call, so the caller sees the
 *   ordering of the context's stream alone (and a call can be captured into a
 *   CUDA graph on that stream).  Calls return once the work is enqueued, except
 *   those that return a host value (documented per call).
 *   Kernel errors surface as PIC_ERR_CUDA at the next call or at pic_sync.
 * Errors: every call returns a pic_status and never aborts; pic_last_error
 *   gives a one-line description.  Arguments are validated before any launch.
 * Threads: one context per host thread / stream at a time.
 */
#ifndef PIC_H
#define PIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pic_ctx pic_ctx;

typedef enum {
  PIC_OK = 0,
  PIC_ERR_ARG = -1,          /* invalid argument (null pointer, size, order, ...) */
  PIC_ERR_UNSUPPORTED = -2,  /* valid but not implemented (e.g. grid size not a power of two) */
  PIC_ERR_NOMEM = -3,        /* device allocation failed */
  PIC_ERR_CUDA = -4,         /* a CUDA call or kernel failed */
  PIC_ERR_CAPACITY = -5,     /* more particles than the context was sized for */
  PIC_ERR_TIMEOUT = -6,      /* a bounded device-side wait (for a bulk copy) gave up; reported by pic_sync */
  PIC_ERR_NONFINITE = -7     /* reserved: non-finite values detected */
} pic_status;

typedef enum {
  PIC_PSATD_STANDARD = 0,          /* Sec. 4.2, Eqs. eq_update_B/E_with_rho_standard */
  PIC_PSATD_GALILEAN = 1,          /* Sec. 4.3, Eqs. eq_update_B/E_with_rho_galilean */
  PIC_PSATD_AVERAGED_GALILEAN = 2  /* Sec. 4.4, Eqs. eq_update_B/E_with_rho_averaged */
} pic_variant;

typedef enum {
  PIC_FP64 = 0,  /* plain FP64 form: every array double, FP64 arithmetic */
  PIC_FP32 = 1   /* FP32 form: FP32 fields, particles and FFTs; FP64 coefficient tables and diagnostics */
} pic_precision;

typedef enum {
  PIC_PUSHER_BORIS = 0,  /* Boris rotation (the default) */
  PIC_PUSHER_VAY = 1     /* Vay's pusher, used for the paper's runs (Secs. 5.2-5.3) */
} pic_pusher;

typedef enum {
  PIC_CYCLE_HYBRID = 0,  /* the hybrid nodal-staggered cycle of Sec. 2 (the method) */
  PIC_CYCLE_NODAL = 1,   /* the nodal comparison cycle of Sec. 2: every quantity on the nodes,
                            [k]_c in the solver, no centering */
  PIC_CYCLE_STAGGERED = 2, /* the staggered comparison cycle of Sec. 2: the Yee-grid solver, E, B
                              gathered from and J deposited at their own Yee positions, no centering */
  PIC_CYCLE_HYBRID_FDTD = 3 /* the hybrid scheme with an FDTD solver (the adaptation to FDTD the
                               conclusions of Sec. 6 state): nodal gather / deposit and the
                               finite-order centering of Sec. 3 around a Yee finite-difference
                               update of order 2m, no Fourier transforms */
} pic_cycle;

/*
 * Optional extension block (pass NULL for defaults).  struct_size must be
 * sizeof(pic_ext) of the caller's header (versioning).
 *   spectral_order[3]: order 2m of the modified wave numbers [k]_s, [k]_c of
 *     Sec. 4.1 per axis; 0 = infinite order ([k] = k).  Default 0.
 *   precision: PIC_FP64 (the pic_step family) or PIC_FP32 (the pic_step32 family).
 *   c, eps0: speed of light and vacuum permittivity.  Defaults 1, 1.
 *   tile[3]: particle tile edge in cells per axis for binning (powers of two
 *     dividing the grid).  Default 8, 8, 8.
 *   sort_interval: re-bin the particles every this many steps inside pic_step
 *     (0 = never).  Default 20.
 *   cuda_stream: a cudaStream_t; NULL = legacy default stream.
 *   filter_passes: passes of the bilinear (1/4, 1/2, 1/4) smoothing filter applied
 *     along every axis to the deposited J and rho before the field solve (Sec. 2),
 *     0..8; applied in Fourier space as prod_a cos^2(k_a dx_a / 2) per pass to J,
 *     rho^n and rho^{n+1} inside the step (the rho array keeps the unfiltered
 *     deposit; the J written back is the filtered, Yee-centered one).  Default 0.
 *   pusher: pic_pusher.  Default PIC_PUSHER_BORIS.
 *   cycle: pic_cycle.  With PIC_CYCLE_NODAL the caller's E, B and the J written back
 *     live on the nodes (no Yee offsets), the solver uses [k]_c in place of [k]_s (with
 *     the Nyquist entry 0 at infinite order, the centered derivative of node-based data)
 *     and zeta_F = 1.  With PIC_CYCLE_STAGGERED the fields stay on the Yee grid throughout:
 *     the shapes of each component are taken on its own staggered grid (offset 1/2 cell
 *     along its staggered axes) for the gather of E, B and the deposit of J (rho nodal), and
 *     zeta_F = 1.  The FP32 form then uses the untiled push.  With PIC_CYCLE_HYBRID_FDTD
 *     the fields advance in real space on the Yee grid by leapfrog with the B update split
 *     in halves (B^{n+1/2} = B^n - (dt/2) curl E^n; E^{n+1} = E^n + dt (c^2 curl B^{n+1/2}
 *     - J^{n+1/2} / eps0); B^{n+1} = B^{n+1/2} - (dt/2) curl E^{n+1}), each derivative the
 *     staggered difference sum_n c_n (f_{j+n} - f_{j-n+1}) / dx with c_n = alpha^s_{m,n} /
 *     (2n - 1), 2m = spectral_order of the axis (0 means 2: Yee's scheme; at most 32), whose symbol is
 *     i [k]_s.  E, B are centered to the nodes and J to the Yee grid by the stencils of Sec. 3
 *     (Eq. staggered_finite_sum) in real space; filter_passes smooths the nodal J in real
 *     space before its centering.  rho is deposited (rho^{n+1} on exit) but the solver does
 *     not use it.  Both precisions (pic_step, pic_step32).  Requires PIC_PSATD_STANDARD
 *     (PIC_ERR_UNSUPPORTED otherwise) and dt within the Courant limit
 *     c dt sqrt(sum_a max_k [k_a]_s^2) <= 2 (PIC_ERR_ARG otherwise).  Default PIC_CYCLE_HYBRID.
 *   reserved: must be 0.
 */
typedef struct {
  uint32_t struct_size;
  int32_t spectral_order[3];
  int32_t precision;
  double c;
  double eps0;
  int32_t tile[3];
  int32_t sort_interval;
  void* cuda_stream;
  int32_t filter_passes;
  int32_t pusher;
  int32_t cycle;
  int32_t reserved;
} pic_ext;

/* Fill *ext with the defaults listed above. */
void pic_ext_default(pic_ext* ext);

/*
 * pic_init: create a context for one grid and method configuration.
 *   grid[3]             Nx, Ny, Nz (powers of two in [8, 1024]; else PIC_ERR_UNSUPPORTED).
 *   dx[3]               cell sizes (> 0).
 *   dt                  time step (> 0).
 *   shape_order         particle shape: 1 (CIC), 2 (quadratic), 3 (cubic) B-spline
 *                       on the nodal grid (Secs. 5.2-5.3 use cubic splines).
 *   centering_order[3]  order 2m of the finite-order centering of Sec. 3 per axis
 *                       (even, 2 <= 2m <= 32 and 2m <= N).
 *   psatd_variant       a pic_variant.
 *   v_gal[3]            Galilean velocity (ignored by PIC_PSATD_STANDARD; |v_gal| < c).
 *   ext                 NULL or a pic_ext.
 * Allocates the work buffers and builds the per-mode FP64 coefficient tables
 * of Sec. 4 on the device.  On success *out is a new context (free it with
 * pic_destroy); on failure *out is NULL.  Synchronous.
 */
pic_status pic_init(pic_ctx** out, const int64_t grid[3], const double dx[3], double dt,
                    int shape_order, const int32_t centering_order[3], int psatd_variant,
                    const double v_gal[3], const pic_ext* ext);

void pic_destroy(pic_ctx* ctx);

/* Last error message of this context (static storage owned by the context). */
const char* pic_last_error(const pic_ctx* ctx);

/* Wait for the context's stream; returns PIC_ERR_CUDA if any enqueued work failed, and
 * PIC_ERR_TIMEOUT (once, the flag is cleared) if a kernel's bounded wait for one of its bulk
 * copies gave up since the last pic_sync (the kernel then skipped its work: results are invalid). */
pic_status pic_sync(pic_ctx* ctx);

/*
 * One particle species, device SoA of n particles (FP64 form).
 *   x, y, z    positions in [0, N dx) per axis (Galilean coordinates for the
 *              Galilean variants).
 *   ux, uy, uz momentum per unit mass u = gamma v, at the half step u^{n-1/2}.
 *   w          macro-particle weight (number of physical particles).
 *   id         optional (may be NULL): an int64 tag per particle, permuted
 *              together with the other arrays when the library re-bins.
 *   q, m       charge and mass of one physical particle.
 * The library may PERMUTE all arrays of a species in place (tile binning);
 * the multiset of particles is unchanged.
 */
typedef struct {
  int64_t n;
  double q;
  double m;
  double* x;
  double* y;
  double* z;
  double* ux;
  double* uy;
  double* uz;
  double* w;
  int64_t* id;
} pic_species;

/*
 * pic_step: advance fields and particles by nsteps hybrid PIC steps (Sec. 2).
 *   E[3], B[3]  in/out: Yee-grid fields at t^n on entry, t^{n+nsteps} on exit.
 *   J[3]        out: J^{n+nsteps-1/2} on the Yee grid (centered from the nodal deposit), or
 *               J = NULL when the caller does not need it (saves the three transforms of J).
 *   rho         in/out: nodal rho^n on entry (see pic_deposit_rho), rho^{n+nsteps} on exit.
 *   sp          n_species species (positions x^n, momenta u^{n-1/2} on entry).
 * Per step: gather at x^n from the nodal E, B (Sec. 2); Boris push; move by
 * dt (v - v_gal); direct deposition of J^{n+1/2} at x^{n+1/2} = (x^n + x^{n+1})/2
 * and of rho^{n+1} at x^{n+1} (nodal); centering of J to the Yee grid (Sec. 3);
 * PSATD update in Fourier space (Sec. 4); centering of E, B to the nodal grid.
 * The centering stencils are applied as their exact Fourier symbol (App. C,
 * zeta_F) inside the k-space update.  Averaged Galilean: the fields gathered at
 * step n+1 are <E>^{n+1}, <B>^{n+1} (Sec. 4.4); the first step of each call
 * gathers E, B.  Asynchronous.
 */
pic_status pic_step(pic_ctx* ctx, double* const E[3], double* const B[3], double* const J[3],
                    double* rho, const pic_species* sp, int n_species, int nsteps);

/*
 * Per-particle adjoint arrays of one species (reverse mode): adjoints of the
 * positions x, y, z and momenta ux, uy, uz, device FP64 arrays of n elements,
 * index-aligned with the species they belong to.
 */
typedef struct {
  int64_t n;
  double* x;
  double* y;
  double* z;
  double* ux;
  double* uy;
  double* uz;
} pic_species_adjoint;

/*
 * pic_adjoint_step: reverse mode of one pic_step (FP64 form; standard and
 * Galilean variants).  The paper states the forward method only; the reverse
 * applies the transpose of each map of the hybrid cycle in reverse order:
 * the PSATD update of Sec. 4 (per mode, the conjugate transpose of its
 * coefficient matrix), the centering of Sec. 3 (transposes), the direct
 * deposits and the gather (transposes of each other, plus the B-spline
 * derivative for the positions), x^{n+1} = x^n + dt (v - v_gal), v = u/gamma
 * and the Boris push.
 *   E[3], B[3]     the forward Yee fields at t^n (read only).
 *   sp             the forward particles at t^n: x^n, u^{n-1/2} (read only, never permuted).
 *   Ebar[3], Bbar[3], rhobar   in: adjoints of E^{n+1}, B^{n+1} (Yee) and rho^{n+1} (nodal);
 *                  out: adjoints of E^n, B^n and rho^n.
 *   spbar          per species, in: adjoints of x^{n+1}, u^{n+1/2}; out: of x^n, u^{n-1/2}.
 * The caller keeps checkpoints of the forward state and recomputes each step's
 * state before reversing it (pic_step must then run with sort_interval = 0 so
 * that particle order is stable).  PIC_ERR_UNSUPPORTED for the averaged variant,
 * the Vay pusher, filter_passes > 0 and the nodal cycle.  Asynchronous.
 */
pic_status pic_adjoint_step(pic_ctx* ctx, const double* const E[3], const double* const B[3],
                            const pic_species* sp, int n_species, double* const Ebar[3], double* const Bbar[3],
                            double* rhobar, const pic_species_adjoint* spbar);

/*
 * pic_field_energy_adjoint: the adjoint seed of the probe-box field energy, the loss of the
 * reverse mode.  W = 1/2 sum (eps0 |E|^2 + |B|^2 / mu0) dV over the cells with index in
 * [box_lo, box_hi) per axis of each Yee component (Sec. 2 (iii)), so
 *   Ebar[c] = scale * eps0 dV E[c],  Bbar[c] = scale * dV B[c] / mu0  inside the box, 0 outside,
 * with 1 / mu0 = eps0 c^2; scale is the gradient arriving from above (1 for dW itself).
 *   E[3], B[3]        Yee fields (device, read only).
 *   box_lo, box_hi    HOST int64[3] each, or both NULL for the whole grid (PIC_ERR_ARG for one
 *                     NULL or a box outside [0, N)).
 *   Ebar[3], Bbar[3]  device, overwritten over the whole grid; they must not overlap E or B.
 * FP64 contexts only (PIC_ERR_ARG otherwise).  Asynchronous.
 */
pic_status pic_field_energy_adjoint(pic_ctx* ctx, const double* const E[3], const double* const B[3],
                                    const int64_t box_lo[3], const int64_t box_hi[3], double scale,
                                    double* const Ebar[3], double* const Bbar[3]);

/*
 * pic_deposit_rho: rho (nodal, overwritten) = sum over species of the direct
 * charge deposition q w S(x - x_i) / dV at the current positions; use it to
 * form rho^0 before the first pic_step.  Asynchronous.
 */
pic_status pic_deposit_rho(pic_ctx* ctx, const pic_species* sp, int n_species, double* rho);

/*
 * pic_push_deposit: one particle stage in isolation (gather + Boris + move +
 * deposit) from caller-provided NODAL fields En[3], Bn[3]; J_nodal[3] and
 * rho_nodal are overwritten with J^{n+1/2} and rho^{n+1} (nodal).  Particles
 * are updated in place and not re-binned.  Asynchronous.
 */
pic_status pic_push_deposit(pic_ctx* ctx, const double* const En[3], const double* const Bn[3],
                            const pic_species* sp, int n_species, double* const J_nodal[3],
                            double* rho_nodal);

/*
 * pic_bin: tile binning of one species (spec design; the paper is silent).
 * cell_a = floor(x_a * (1/dx_a)) mod N_a, tile_a = cell_a / tile_edge_a,
 * tile id = (tile_x * nty + tile_y) * ntz + tile_z.  Permutes the species
 * arrays in place so that tile ids are non-decreasing, and writes
 * offsets[n_tiles + 1] (int64, device, exclusive prefix sum of the per-tile
 * counts) if offsets is not NULL.  The order inside a tile is unspecified.
 * n_tiles = prod(N_a / tile_edge_a).  Asynchronous.
 */
pic_status pic_bin(pic_ctx* ctx, const pic_species* sp, int64_t* offsets);

/* Number of tiles of the context's tiling. */
int64_t pic_num_tiles(const pic_ctx* ctx);

/*
 * pic_center_to_nodal: finite-order centering of the six Yee components
 * F = {E^x, E^y, E^z, B^x, B^y, B^z} onto the nodal grid, as real-space stencils
 * (Sec. 3, Eq. staggered_finite_sum) applied along each staggered axis of each
 * component in x, y, z order, periodic wrap.  out[6] nodal, overwritten.  No out[c] may
 * overlap any F[c'] or another out[c'] (a stencil pass would read neighbours it has already
 * overwritten): such calls return PIC_ERR_ARG.
 * Asynchronous.
 */
pic_status pic_center_to_nodal(pic_ctx* ctx, const double* const F[6], double* const out[6]);

/*
 * pic_center_to_yee: finite-order centering of nodal J^x, J^y, J^z onto their
 * Yee positions, the mirror image of Eq. staggered_finite_sum:
 * f_{j+1/2} = sum_n alpha^s_{m,n} (f_{j+n} + f_{j-n+1}) / 2 along the staggered
 * axis of each component.  out[3] overwritten; no out[c] may overlap any Jn[c'] or another
 * out[c'] (PIC_ERR_ARG).  Asynchronous.
 */
pic_status pic_center_to_yee(pic_ctx* ctx, const double* const Jn[3], double* const out[3]);

/*
 * pic_fft_forward / pic_fft_inverse: 3D real-to-complex DFT of ncomp real
 * arrays (App. A.1, Eq. Fourier_discrete, without the half-cell phase) and its
 * unnormalised inverse (complex-to-real; the imaginary parts of the k_z = 0 and
 * k_z = Nyquist planes are ignored).  spec[c] points to a complex array of
 * Nx*Ny*(Nz/2+1) (re, im) double pairs.  The inverse overwrites spec.
 * 1 <= ncomp <= 6.  Asynchronous.
 */
pic_status pic_fft_forward(pic_ctx* ctx, const double* const real[], double* const spec[], int ncomp);
pic_status pic_fft_inverse(pic_ctx* ctx, double* const spec[], double* const real[], int ncomp);

/*
 * pic_maxwell_step: the field solve of one step in isolation (Sec. 4):
 * Yee E^n, B^n, J^{n+1/2} (Yee), rho^n, rho^{n+1} (nodal) -> Yee E^{n+1}, B^{n+1}
 * (in place).  For the averaged variant, Eavg[3], Bavg[3] (may be NULL for the
 * other variants) receive <E>^{n+1}, <B>^{n+1} at the Yee positions.
 * On a PIC_CYCLE_HYBRID_FDTD context this is the finite-difference leapfrog step
 * described under pic_ext.cycle; rho_n and rho_np1 are not read and may be NULL.
 * Asynchronous.
 */
pic_status pic_maxwell_step(pic_ctx* ctx, double* const E[3], double* const B[3],
                            const double* const J[3], const double* rho_n,
                            const double* rho_np1, double* const Eavg[3], double* const Bavg[3]);

/*
 * pic_coefficient: copy one per-mode coefficient table (complex, layout of the
 * spectral arrays) into out (device, Nx*Ny*(Nz/2+1) (re, im) pairs).  Names:
 * "TC" = theta_c^2 C, "TS" = theta_c^2 S/omega_s, "X1", "X2", "TX3" = theta_c^2 X3,
 * "X4" (Secs. 4.2-4.3), and for the averaged variant "Psi1", "Psi2", "Y1", "Y2",
 * "Y3", "Y4" (Sec. 4.4).  Unknown name: PIC_ERR_ARG.  Asynchronous.
 */
pic_status pic_coefficient(pic_ctx* ctx, const char* name, double* out);

/*
 * pic_field_energy: W = 1/2 sum (eps0 |E|^2 + |B|^2 / mu0) dV over the cells with
 * index in [box_lo, box_hi) per axis of each Yee component (Sec. 2 (iii); NULL
 * box = whole grid), FP64 reduction; *out is a HOST double.  Synchronous.
 */
pic_status pic_field_energy(pic_ctx* ctx, const double* const E[3], const double* const B[3],
                            const int64_t box_lo[3], const int64_t box_hi[3], double* out);

/* pic_total_charge: sum(rho) dV of a nodal array; *out is a HOST double.  Synchronous. */
pic_status pic_total_charge(pic_ctx* ctx, const double* rho, double* out);

/*
 * ---------------------------------------------------------------------------
 * FP32 form (contexts created with precision = PIC_FP32).  Same step, same
 * readings of the paper; fields, particles, deposits and FFTs in FP32; the PSATD
 * coefficient tables stay FP64 (rounded to FP32 at use) and the energy / charge
 * reductions accumulate in FP64.  Calling an FP32 entry point on an FP64
 * context (or the reverse) returns PIC_ERR_ARG.
 * ---------------------------------------------------------------------------
 *
 * One species in the FP32 form, device SoA of n particles.
 *   cell       int32 linear index (ix * Ny + iy) * Nz + iz of the cell holding
 *              the particle (node (ix, iy, iz) is its lower corner).
 *   fx, fy, fz FP32 offsets in [0, 1) inside that cell, in units of the cell size:
 *              position x = (ix + fx) dx, etc.
 *   ux, uy, uz, w, id, q, m: as in pic_species (FP32 arrays; id optional).
 * Arrays may be permuted in place by binning, as in the FP64 form.
 */
typedef struct {
  int64_t n;
  double q;
  double m;
  int32_t* cell;
  float* fx;
  float* fy;
  float* fz;
  float* ux;
  float* uy;
  float* uz;
  float* w;
  int64_t* id;
} pic_species32;

/* pic_step32: pic_step in the FP32 form; E, B, J (Yee) and rho (nodal) are float arrays. */
pic_status pic_step32(pic_ctx* ctx, float* const E[3], float* const B[3], float* const J[3], float* rho,
                      const pic_species32* sp, int n_species, int nsteps);

/* pic_deposit_rho32: pic_deposit_rho in the FP32 form. */
pic_status pic_deposit_rho32(pic_ctx* ctx, const pic_species32* sp, int n_species, float* rho);

/* pic_push_deposit32: pic_push_deposit in the FP32 form (nodal float fields in, nodal float J, rho out). */
pic_status pic_push_deposit32(pic_ctx* ctx, const float* const En[3], const float* const Bn[3],
                              const pic_species32* sp, int n_species, float* const J_nodal[3], float* rho_nodal);

/* pic_bin32: pic_bin in the FP32 form (tile from the integer cell index).  Inside a tile the
 * particles come out ordered by cell, z fastest, then x, then y (the order the tiled push's
 * shared-memory layout is built for); the order among particles of one cell is unspecified. */
pic_status pic_bin32(pic_ctx* ctx, const pic_species32* sp, int64_t* offsets);

/* pic_fft_forward32 / pic_fft_inverse32: pic_fft_forward / inverse on float arrays
 * (spectra: Nx*Ny*(Nz/2+1) (re, im) float pairs). */
pic_status pic_fft_forward32(pic_ctx* ctx, const float* const real[], float* const spec[], int ncomp);
pic_status pic_fft_inverse32(pic_ctx* ctx, float* const spec[], float* const real[], int ncomp);

/* pic_field_energy32 / pic_total_charge32: FP64 reductions over float arrays (HOST results). */
pic_status pic_field_energy32(pic_ctx* ctx, const float* const E[3], const float* const B[3],
                              const int64_t box_lo[3], const int64_t box_hi[3], double* out);
pic_status pic_total_charge32(pic_ctx* ctx, const float* rho, double* out);

/*
 * pic_species32_from_species: FP64 species -> FP32-form species, on the device.  Per
 * coordinate, with t = x * (1/dx) rounded to FP64 (the multiply of the FP64 form's cell rule),
 * cell index i = floor(t) and offset f = t - i (exact in FP64) rounded once to FP32; an offset
 * that rounds to 1.0 becomes offset 0 of the next cell; the cell wraps into [0, N).  cell =
 * (ix * Ny + iy) * Nz + iz.  ux, uy, uz, w are rounded to FP32; id is copied when both sides give
 * one (PIC_ERR_ARG when only one does).  in->n must equal out->n; out's arrays are overwritten
 * and must not overlap in's.  The paper holds positions in floating point only: the (cell,
 * offset) form is the FP32 form's own representation.  Any context precision (only the grid and
 * dx are used).  Asynchronous.
 */
pic_status pic_species32_from_species(pic_ctx* ctx, const pic_species* in, const pic_species32* out);

/*
 * pic_species32_to_species: the reverse: x = (i + f) dx in FP64 (i + f is exact), u and w
 * widened to FP64, id copied as above.  Asynchronous.
 */
pic_status pic_species32_to_species(pic_ctx* ctx, const pic_species32* in, const pic_species* out);

/*
 * ---- Diagnostics (not on the step's hot path; FP64 arithmetic; HOST results) ----
 *
 * pic_stencil_extent: stencil extent of the coefficient table `coef` (names as in
 * pic_coefficient) along axis 0, 1 or 2 (Sec. 2 (ii), Eq. stencil_extent): the
 * modulus of the inverse DFT of the table along the axis, averaged over the Fourier
 * indices of the two other axes (over their full range: the stored half spectrum is
 * extended by g(-k) = conj g(k)).  out: HOST, N_axis doubles, out[j] = Gamma(j dx_axis)
 * (periodic: j > N/2 are the offsets j - N).  Any context precision.  Synchronous.
 */
pic_status pic_stencil_extent(pic_ctx* ctx, const char* coef, int axis, double* out);

/*
 * pic_axis_tables: the 1D tables of axis a used by the update, HOST copies of N_a
 * doubles each in FFT order (k_j = 2 pi m_j / (N_a dx_a), m_j the signed index with the
 * Nyquist index at -N_a/2): ks = [k]_s and kc = [k]_c at the context's spectral order
 * (Sec. 4.1, Eqs. k_staggered / k_centered) and zeta = zeta_F, the Fourier symbol of the
 * centering of order centering_order[a] (App. C).  Nodal cycle: ks = kc = the solver's
 * [k]_c and zeta = 1; staggered cycle: zeta = 1; FDTD cycle: ks = the symbol of the
 * finite difference (order 2 when spectral_order is 0).  Any pointer may be NULL.  Synchronous.
 */
pic_status pic_axis_tables(pic_ctx* ctx, int axis, double* ks, double* kc, double* zeta);

/*
 * pic_vacuum_dispersion: numerical vacuum frequency of the context's update for waves
 * along axis a (Sec. 2 (i), App. B): per Fourier index along the axis (the other two
 * indices 0) the transverse block of the update, [[TC, -i c^2 TS [k]_s], [-i TS [k]_s, TC]],
 * has eigenvalues TC +- i c TS [k]_s; omega = (larger eigenvalue phase) / dt.  Standard
 * PSATD gives omega = c |[k]_s|; Galilean phases are shifted by Omega_c dt.  FDTD cycle:
 * the leapfrog's omega = (2 / dt) asin(c dt |[k]_s| / 2).  omega: HOST, N_a doubles, FFT
 * order.  Synchronous.
 */
pic_status pic_vacuum_dispersion(pic_ctx* ctx, int axis, double* omega);

/*
 * pic_beam_rms / pic_beam_rms32: averaged transverse RMS size of a species (Sec. 5.3,
 * Eq. RMS_pwfa): delta = 1/2 sqrt(sum w (x - <x>)^2 / sum w) + 1/2 sqrt(sum w (y - <y>)^2
 * / sum w), <.> the w-weighted means, positions as stored (no periodic unwrapping; FP32
 * form: x = (ix + fx) dx in FP64).  delta: HOST.  PIC_ERR_ARG for an empty species or a
 * non-positive weight sum.  Synchronous.
 */
pic_status pic_beam_rms(pic_ctx* ctx, const pic_species* sp, double* delta);
pic_status pic_beam_rms32(pic_ctx* ctx, const pic_species32* sp, double* delta);


/*
 * pic_center_to_nodal_static: the same centering as pic_center_to_nodal, for
 * callers that cannot allocate device memory.  The paper has no counterpart;
 * this exists for host programs that own every byte of device memory through
 * their own pool and forbid other allocations, and for loops where the device
 * synchronisation implied by cudaMalloc / cudaFree is not acceptable.  Such
 * callers cannot create a pic_ctx (pic_init allocates), so this entry point
 * takes the grid and orders directly and allocates nothing: it calls no
 * cudaMalloc, cudaFree or allocating library routine.
 *   grid[3]             Nx, Ny, Nz: powers of two in [2, 1024], with
 *                       Nx * Ny * Nz <= 2,097,152 (2^21) cells, else PIC_ERR_CAPACITY.
 *   centering_order[3]  as in pic_init.
 *   F[6], out[6]        device arrays as in pic_center_to_nodal (caller-owned); no out[c]
 *                       may overlap any F[c'] or another out[c'] (PIC_ERR_ARG).
 *   cuda_stream         a cudaStream_t, or NULL for the legacy default stream.
 * Its scratch (the intermediate of the two-axis centering of B^x, B^y, B^z) is a
 * file-scope static device array of 2^21 doubles (16 MiB) that every GPU which
 * loads the library holds until the process exits.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress) with the device
 * current; make that first call before any stream capture.  All calls share the
 * one array: calls that overlap on the GPU (different streams, or different host
 * threads, without ordering between them) race on it.  Every element the
 * scratch is read from is written first in the same call, so no clearing is
 * needed.  Errors: PIC_ERR_ARG / PIC_ERR_UNSUPPORTED (bad arguments),
 * PIC_ERR_CAPACITY (grid larger than the scratch; a message goes to stderr),
 * PIC_ERR_CUDA (no current device or a failed launch).  Asynchronous.
 */
pic_status pic_center_to_nodal_static(const int64_t grid[3], const int32_t centering_order[3],
                                      const double* const F[6], double* const out[6], void* cuda_stream);

/*
 * pic_timing: enable (1) or disable (0) per-stage device timing and reset the
 * accumulators.  When enabled, each stage call of pic_step records a pair of
 * CUDA events on the context stream.  Stages: "push" (gather + Boris + deposit),
 * "fft", "update" (fused PSATD k-space update), "bin" (tile binning), "other"
 * (phase, centering-symbol and diagnostic kernels).  Kernel launches are
 * counted per stage whether or not timing is enabled.  Synchronous.
 */
pic_status pic_timing(pic_ctx* ctx, int enable);

/*
 * pic_timing_read: total device time in ms (*ms, HOST) and kernel launches
 * (*launches, HOST) of one stage since the last pic_timing call; stage "all"
 * gives the launch total and the summed time.  Synchronous.
 */
pic_status pic_timing_read(pic_ctx* ctx, const char* stage, double* ms, int64_t* launches);

#ifdef __cplusplus
}
#endif

#endif /* PIC_H */
