// PSATD coefficient tables and the fused k-space update (Sec. 4).
//
// Per-mode coefficients are built once, on the device, in FP64.  The paper's
// closed forms (Secs. 4.2-4.4) are 0/0 at omega_s = 0 and Omega_c = 0 and lose
// digits near those points and near omega_s = |Omega_c|, so every coefficient
// is evaluated from an equivalent integral representation of the analytic
// solution (the same ODE the paper integrates in App. A):
//   K1(phi, a) = int_0^1 sigma sinc(phi sigma) e^{i a sigma} d sigma        (X1 = dt^2/eps0 K1)
//   K2(phi, a) = (K1(phi,a) - e^{ia} K1(phi,0)) / (1 - e^{ia})               (X2 = c^2 dt^2/eps0 K2)
//   K3(phi, a) = e^{ia} (K1(phi,a) - K1(phi,0)) / (1 - e^{ia})              (theta^2 X3 = c^2 dt^2/eps0 K3)
// with phi = omega_s dt, a = Omega_c dt, and for the averaged fields the time
// average over [t^{n+1/2}, t^{n+3/2}] of the same solution.  Where the closed
// forms in terms of E(b) = int_0^1 e^{ib s} ds, F(b) = int_{1/2}^{3/2} e^{ib s} ds
// and H(b) = int_{1/2}^{3/2} int_0^s e^{ibu} du ds are well conditioned
// (phi >= 0.3 and |a| >= 0.3) they are used; elsewhere the integrals are taken
// by 16-point Gauss-Legendre quadrature of stable integrands (entire functions
// of modest frequency, so the rule is exact to rounding).  a = 0 uses the
// standard forms (Sec. 4.2) directly.
#include "pic_internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace {

constexpr int kGL = 16;
struct GaussLegendre {
  double x[kGL];  // nodes on [0, 1]
  double w[kGL];  // weights, sum 1
};

// ---------------------------------------------------------------------------
// scalar helpers (device)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double sinc_d(double x) {
  const double ax = fabs(x);
  if (ax < 1e-3) {
    const double x2 = x * x;
    return 1.0 - x2 * (1.0 / 6.0) + x2 * x2 * (1.0 / 120.0);
  }
  return sin(x) / x;
}
__device__ __forceinline__ double2 cis(double t) {
  double s, c;
  sincos(t, &s, &c);
  return make_double2(c, s);
}
// (x - sin x) / x^3
__device__ double k2s(double x) {
  if (fabs(x) < 0.5) {
    const double x2 = x * x;
    double term = 1.0 / 6.0, sum = term;
    for (int n = 2; n <= 12; ++n) {  // (-1)^{n+1} x^{2n-2} / (2n+1)!
      term *= -x2 / ((2.0 * n) * (2.0 * n + 1.0));
      sum += term;
    }
    return sum;
  }
  return (x - sin(x)) / (x * x * x);
}
// (x cos x - sin x) / x^3
__device__ double k3s(double x) {
  if (fabs(x) < 0.5) {
    const double x2 = x * x;
    // sum_{n>=1} (-1)^n 2n / (2n+1)! x^{2n-2}
    double f = 1.0 / 6.0;  // 1/(2n+1)! at n = 1
    double p = 1.0;        // x^{2n-2}
    double sum = 0.0;
    for (int n = 1; n <= 12; ++n) {
      if (n > 1) {
        f /= (2.0 * n) * (2.0 * n + 1.0);
        p *= x2;
      }
      sum += ((n & 1) ? -1.0 : 1.0) * 2.0 * n * f * p;
    }
    return sum;
  }
  double s, c;
  sincos(x, &s, &c);
  return (x * c - s) / (x * x * x);
}
// K1(phi, 0) = (1 - cos phi) / phi^2 = sinc(phi/2)^2 / 2
__device__ __forceinline__ double k1s(double x) {
  const double s = sinc_d(0.5 * x);
  return 0.5 * s * s;
}
// E(b) = e^{ib/2} sinc(b/2)
__device__ __forceinline__ double2 Eint(double b) { return cscale(cis(0.5 * b), sinc_d(0.5 * b)); }
// F(b) = e^{ib} sinc(b/2)
__device__ __forceinline__ double2 Fint(double b) { return cscale(cis(b), sinc_d(0.5 * b)); }
// H(b) = (F(b) - 1) / (i b); series sum_n (ib)^n / (n+1)! M_{n+1}, M_p = ((3/2)^{p+1} - (1/2)^{p+1})/(p+1)
__device__ double2 Hint(double b) {
  if (fabs(b) < 0.5) {
    double2 p = make_double2(1.0, 0.0);  // (ib)^n / (n+1)!
    double2 sum = make_double2(0.0, 0.0);
    double a3 = 1.5 * 1.5, a1 = 0.25;     // (3/2)^{n+2}, (1/2)^{n+2}
    for (int n = 0; n <= 22; ++n) {
      if (n > 0) {
        p = cscale(cmuli(cscale(p, b)), 1.0 / (n + 1.0));
        a3 *= 1.5;
        a1 *= 0.5;
      }
      const double M = (a3 - a1) / (n + 2.0);
      sum = cadd(sum, cscale(p, M));
    }
    return sum;
  }
  const double2 f = Fint(b);
  return cdiv(make_double2(f.x - 1.0, f.y), make_double2(0.0, b));
}
// h(u) = (e^{iau} - 1) / (e^{ia} - 1) = e^{ia(u-1)/2} u sinc(au/2) / sinc(a/2)
__device__ __forceinline__ double2 hfun(double a, double u) {
  return cscale(cis(0.5 * a * (u - 1.0)), u * sinc_d(0.5 * a * u) / sinc_d(0.5 * a));
}

struct Coefs {
  double2 v[COEF_COUNT];
};

// All coefficients of one mode.  phi = omega_s dt >= 0, a = Omega_c dt.
__device__ Coefs mode_coefs(double phi, double a, bool averaged, double dt, double c, double eps0,
                            const GaussLegendre& gl) {
  Coefs r;
  const double dt2e = dt * dt / eps0, c2dt2e = c * c * dt * dt / eps0;
  const double sphi = sinc_d(phi), cphi = cos(phi);
  const bool wc = phi >= 0.3 && fabs(a) >= 0.3;
  double2 K1, K2, K3;
  const double2 ea = cis(a);
  if (a == 0.0) {
    K1 = make_double2(k1s(phi), 0.0);
    K2 = make_double2(k2s(phi), 0.0);
    K3 = make_double2(k3s(phi), 0.0);
  } else if (wc) {
    K1 = cdiv(csub(Eint(a + phi), Eint(a - phi)), make_double2(0.0, 2.0 * phi));
    const double K10 = k1s(phi);
    const double2 den = make_double2(1.0 - ea.x, -ea.y);
    K2 = cdiv(csub(K1, cscale(ea, K10)), den);
    K3 = cdiv(cmul(ea, make_double2(K1.x - K10, K1.y)), den);
  } else {
    K1 = K2 = K3 = make_double2(0.0, 0.0);
    const double sa = sinc_d(0.5 * a);
    for (int q = 0; q < kGL; ++q) {
      const double s = gl.x[q], w = gl.w[q];
      const double g = s * sinc_d(phi * s);  // sin(phi s) / phi
      K1 = cadd(K1, cscale(cis(a * s), w * g));
      K2 = cadd(K2, cscale(cis(0.5 * a * s), w * g * (1.0 - s) * sinc_d(0.5 * a * (1.0 - s)) / sa));
      K3 = csub(K3, cscale(cis(0.5 * a * (1.0 + s)), w * g * s * sinc_d(0.5 * a * s) / sa));
    }
  }
  r.v[COEF_TC] = cscale(ea, cphi);
  r.v[COEF_TS] = cscale(ea, dt * sphi);
  r.v[COEF_X1] = cscale(K1, dt2e);
  r.v[COEF_X2] = cscale(K2, c2dt2e);
  r.v[COEF_TX3] = cscale(K3, c2dt2e);
  // X4 = (dt/eps0) (i a K1 - e^{ia} sinc phi)
  r.v[COEF_X4] = cscale(csub(cscale(cmuli(K1), a), cscale(ea, sphi)), dt / eps0);
  if (!averaged) return r;

  // averaged fields: <f> = int_{1/2}^{3/2} f(sigma dt) d sigma
  const double2 Psi1 = cscale(cadd(Fint(a + phi), Fint(a - phi)), 0.5);
  const double2 Psi3 = Fint(a);
  double2 Psi2n, Y1n, Qn;  // Psi2 = -dt Psi2n, Y1 = dt^2/eps0 Y1n, <Q> = dt^2 Qn
  if (wc) {
    const double2 den2 = make_double2(0.0, 2.0 * phi);
    Psi2n = cdiv(csub(Fint(a + phi), Fint(a - phi)), den2);
    Y1n = cdiv(csub(Hint(a + phi), Hint(a - phi)), den2);
    const double2 num = csub(cscale(csub(Psi3, Psi1), 1.0 / (phi * phi)), Y1n);
    Qn = cdiv(num, make_double2(ea.x - 1.0, ea.y));
  } else {
    Psi2n = Y1n = Qn = make_double2(0.0, 0.0);
    for (int q = 0; q < kGL; ++q) {
      const double s = 0.5 + gl.x[q], w = gl.w[q];
      Psi2n = cadd(Psi2n, cscale(cis(a * s), w * s * sinc_d(phi * s)));
      double2 R = make_double2(0.0, 0.0), Q = make_double2(0.0, 0.0);
      for (int p = 0; p < kGL; ++p) {
        const double u = s * gl.x[p], wu = s * gl.w[p];
        R = cadd(R, cscale(cis(a * u), wu * u * sinc_d(phi * u)));
        if (a != 0.0) {
          const double d = s - u;
          Q = cadd(Q, cscale(cmul(cis(a * d), hfun(a, u)), wu * d * sinc_d(phi * d)));
        }
      }
      Y1n = cadd(Y1n, cscale(R, w));
      if (a != 0.0) Qn = cadd(Qn, cscale(Q, w));
    }
  }
  double2 Y2, Y3;
  if (a == 0.0) {
    // rho linear in time: Y2 = -i c^2/eps0 <int_0^t G(t-s) s/dt ds>, Y3 = -i c^2/eps0 <int_0^t G (1 - s/dt)>
    double A0 = 0.0, A1 = 0.0;
    for (int q = 0; q < kGL; ++q) {
      const double s = 0.5 + gl.x[q], w = gl.w[q];
      A0 += w * s * s * k1s(phi * s);
      A1 += w * s * s * s * k2s(phi * s);
    }
    Y2 = make_double2(0.0, -c2dt2e * A1);
    Y3 = make_double2(0.0, -c2dt2e * (A0 - A1));
  } else {
    Y2 = cscale(cmuli(Qn), -c2dt2e);
    Y3 = cscale(cmuli(csub(Y1n, Qn)), -c2dt2e);
  }
  r.v[COEF_PSI1] = Psi1;
  r.v[COEF_PSI2] = cscale(Psi2n, -dt);
  r.v[COEF_Y1] = cscale(Y1n, dt2e);
  r.v[COEF_Y2] = Y2;
  r.v[COEF_Y3] = Y3;
  // Y4 = i Omega_c Y1 + Psi2 / eps0 = (dt/eps0) (i a Y1n - Psi2n)
  r.v[COEF_Y4] = cscale(csub(cscale(cmuli(Y1n), a), Psi2n), dt / eps0);
  return r;
}

struct TableArgs {
  const double* ks[3];
  const double* kc[3];
  int64_t Ny, nzh, nmode;
  double vg[3];
  double dt, c, eps0;
  int ncoef;
  int averaged;
  double2* coef;
  GaussLegendre gl;
};

// Mode index m -> (ix, iy, iz) for the [Nx][Ny][Nz/2+1] spectra; 32-bit arithmetic (every context
// has fewer than 2^32 modes), Ny a power of two.
__device__ __forceinline__ void mode_xyz(int64_t m, uint32_t nzh, int lgNy, uint32_t& ix, uint32_t& iy,
                                         uint32_t& iz) {
  const uint32_t mm = (uint32_t)m;
  const uint32_t r = mm / nzh;
  iz = mm - r * nzh;
  iy = r & ((1u << lgNy) - 1u);
  ix = r >> lgNy;
}

__global__ void build_tables_kernel(TableArgs t) {
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= t.nmode) return;
  const int64_t iz = m % t.nzh, r = m / t.nzh;
  const int64_t iy = r % t.Ny, ix = r / t.Ny;
  const double kx = t.ks[0][ix], ky = t.ks[1][iy], kz = t.ks[2][iz];
  const double phi = t.c * sqrt(kx * kx + ky * ky + kz * kz) * t.dt;
  const double a = (t.vg[0] * t.kc[0][ix] + t.vg[1] * t.kc[1][iy] + t.vg[2] * t.kc[2][iz]) * t.dt;
  const Coefs cf = mode_coefs(phi, a, t.averaged != 0, t.dt, t.c, t.eps0, t.gl);
  for (int k = 0; k < t.ncoef; ++k) t.coef[k * t.nmode + m] = cf.v[k];
}

// Compact tables: entry (qx, qy, iz) of the quarter qx <= Nx/2, qy <= Ny/2 is the full table's mode
// (qx, qy, iz); the update reads it for the four modes (+-kx, +-ky, kz).
struct CompactArgs {
  const double2* full;
  double* q;
  float* q32;  // or NULL
  int real, ncoef;
  int64_t Ny, nzh, nqy, nq, nmode;
};

__global__ void compact_tables_kernel(CompactArgs c) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= c.nq) return;
  const int64_t iz = e % c.nzh, r = e / c.nzh;
  const int64_t qy = r % c.nqy, qx = r / c.nqy;
  const int64_t m = (qx * c.Ny + qy) * c.nzh + iz;
  for (int k = 0; k < c.ncoef; ++k) {
    const double2 v = c.full[k * c.nmode + m];
    if (c.real) c.q[k * c.nq + e] = v.x;
    else reinterpret_cast<double2*>(c.q)[k * c.nq + e] = v;
    if (c.q32) {
      if (c.real) c.q32[k * c.nq + e] = (float)v.x;
      else reinterpret_cast<float2*>(c.q32)[k * c.nq + e] = make_float2((float)v.x, (float)v.y);
    }
  }
}

// ---------------------------------------------------------------------------
// fused update
// ---------------------------------------------------------------------------
template <class C>
struct UpdArgs {
  C* EB;                // [6][nmode] in/out
  C* J;                 // [3][nmode] in: DFT of the nodal (or Yee, j_yee) deposit; out: Yee-centered
  const C* rn;          // rho^n
  const C* rp;          // rho^{n+1}
  CoefView coef;        // FP64 in every form
  C* G;                 // [6][nmode] out
  // 1D tables in the data precision (the FP32 form reads FP32 copies of them: converting FP64
  // values per mode would run on this part's slow FP64 pipe)
  using R = decltype(C().x);
  const R* ks[3];
  const R* zt[3];
  const R* flt[3];  // bilinear filter symbols per axis (NULL: no filter)
  const C* hs[3];   // half-cell shifts exp(-i k dx / 2)
  int64_t Ny, nzh, nmode;
  double c2;
  double gscale;
  int g_mode;   // 0: G = Z (E, B) * gscale (nodal DFT); 1: G = shift^+ (E, B) * gscale (Yee DFT)
  int j_yee;    // 1: J already Yee-centered paper-convention spectrum (skip zeta)
  int write_j;  // write the Yee-centered J back
};

// The k-space update of one mode (Secs. 4.2-4.4): E, B in and out (paper-convention spectra),
// J in (the DFT of the nodal deposit, or with j_yee the Yee-centered spectrum) and out (Yee-centered,
// after the optional filter), rho^n, rho^{n+1}; G[6] out = the fields the next gather reads (E, B or
// <E>, <B>) times the centering symbols (g_mode 0) or the half-cell shifts back to the Yee DFT
// (g_mode 1), times gscale.  The FP64 coefficient tables are read in FP64 and rounded to the data
// precision at use.
template <int VAR, class C>
__device__ __forceinline__ void mode_update(const UpdArgs<C>& u, uint32_t ix, uint32_t iy, uint32_t iz,
                                            const C (&cf)[COEF_COUNT], C (&E)[3], C (&B)[3], C (&J)[3], C rn,
                                            C rp, C (&G)[6]) {
  using T = decltype(C().x);
  const T k[3] = {(T)u.ks[0][ix], (T)u.ks[1][iy], (T)u.ks[2][iz]};
  const T zx = (T)u.zt[0][ix], zy = (T)u.zt[1][iy], zz = (T)u.zt[2][iz];
  if (!u.j_yee) {
    J[0] = cscale(J[0], zx);
    J[1] = cscale(J[1], zy);
    J[2] = cscale(J[2], zz);
  }
  if (u.flt[0]) {
    // smoothing of the step's deposits: J^{n+1/2}, rho^n, rho^{n+1}
    const T f = (T)(u.flt[0][ix] * u.flt[1][iy] * u.flt[2][iz]);
#pragma unroll
    for (int a = 0; a < 3; ++a) J[a] = cscale(J[a], f);
    rn = cscale(rn, f);
    rp = cscale(rp, f);
  }
  // [k] x F
  auto cross = [&](const C* F, C* o) {
    o[0] = csub(cscale(F[2], k[1]), cscale(F[1], k[2]));
    o[1] = csub(cscale(F[0], k[2]), cscale(F[2], k[0]));
    o[2] = csub(cscale(F[1], k[0]), cscale(F[0], k[1]));
  };
  C kE[3], kB[3], kJ[3];
  cross(E, kE);
  cross(B, kB);
  cross(J, kJ);
  const C TC = cf[COEF_TC], TS = cf[COEF_TS], X1 = cf[COEF_X1], X2 = cf[COEF_X2], TX3 = cf[COEF_TX3],
          X4 = cf[COEF_X4];
  const T c2 = (T)u.c2;
  // rho term: i (theta^2 X3 rho^n - X2 rho^{n+1})
  const C rterm = cmuli(csub(cmul(TX3, rn), cmul(X2, rp)));
  C En[3], Bn[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    // B^{n+1} = TC B - i TS [k]xE + i X1 [k]xJ
    Bn[a] = cadd(cmul(TC, B[a]), cmuli(csub(cmul(X1, kJ[a]), cmul(TS, kE[a]))));
    // E^{n+1} = TC E + i c^2 TS [k]xB + X4 J + rterm [k]
    En[a] = cadd(cadd(cmul(TC, E[a]), cmuli(cscale(cmul(TS, kB[a]), c2))),
                 cadd(cmul(X4, J[a]), cscale(rterm, k[a])));
  }
  C Ga[3], Gb[3];
  if (VAR == 2) {
    const C P1 = cf[COEF_PSI1], P2 = cf[COEF_PSI2], Y1 = cf[COEF_Y1], Y2 = cf[COEF_Y2], Y3 = cf[COEF_Y3],
            Y4 = cf[COEF_Y4];
    const C yr = cadd(cmul(Y3, rn), cmul(Y2, rp));
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      // <B> = Psi1 B + i Psi2 [k]xE + i Y1 [k]xJ
      Gb[a] = cadd(cmul(P1, B[a]), cmuli(cadd(cmul(P2, kE[a]), cmul(Y1, kJ[a]))));
      // <E> = Psi1 E - i c^2 Psi2 [k]xB + Y4 J + (Y3 rho^n + Y2 rho^{n+1}) [k]
      Ga[a] = cadd(csub(cmul(P1, E[a]), cmuli(cscale(cmul(P2, kB[a]), c2))),
                   cadd(cmul(Y4, J[a]), cscale(yr, k[a])));
    }
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Ga[a] = En[a];
      Gb[a] = Bn[a];
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    E[a] = En[a];
    B[a] = Bn[a];
  }
  const T s = (T)u.gscale;
  if (u.g_mode == 0) {
    G[0] = cscale(Ga[0], zx * s);
    G[1] = cscale(Ga[1], zy * s);
    G[2] = cscale(Ga[2], zz * s);
    G[3] = cscale(Gb[0], zy * zz * s);
    G[4] = cscale(Gb[1], zx * zz * s);
    G[5] = cscale(Gb[2], zx * zy * s);
  } else {
    const C hx = cconj(u.hs[0][ix]), hy = cconj(u.hs[1][iy]), hz = cconj(u.hs[2][iz]);
    G[0] = cscale(cmul(Ga[0], hx), s);
    G[1] = cscale(cmul(Ga[1], hy), s);
    G[2] = cscale(cmul(Ga[2], hz), s);
    G[3] = cscale(cmul(Gb[0], cmul(hy, hz)), s);
    G[4] = cscale(cmul(Gb[1], cmul(hx, hz)), s);
    G[5] = cscale(cmul(Gb[2], cmul(hx, hy)), s);
  }
}

// load E, B, J, rho of mode m, update it with the coefficients cf, store E, B (J) and G
template <int VAR, class C>
__device__ __forceinline__ void update_one(const UpdArgs<C>& u, int64_t m, uint32_t ix, uint32_t iy, uint32_t iz,
                                           const C (&cf)[COEF_COUNT]) {
  const int64_t nm = u.nmode;
  C E[3], B[3], J[3], G[6];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    E[a] = u.EB[a * nm + m];
    B[a] = u.EB[(3 + a) * nm + m];
    J[a] = u.J[a * nm + m];
  }
  mode_update<VAR>(u, ix, iy, iz, cf, E, B, J, u.rn[m], u.rp[m], G);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    u.EB[a * nm + m] = E[a];
    u.EB[(3 + a) * nm + m] = B[a];
  }
  if (u.write_j) {
#pragma unroll
    for (int a = 0; a < 3; ++a) u.J[a * nm + m] = J[a];
  }
#pragma unroll
  for (int c = 0; c < 6; ++c) u.G[c * nm + m] = G[c];
}

// One mode per thread over the whole spectrum, coefficients from the full tables.
template <int VAR, class C>
__global__ void __launch_bounds__(256) update_kernel(UpdArgs<C> u) {
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= u.nmode) return;
  uint32_t ix, iy, iz;
  mode_xyz(m, (uint32_t)u.nzh, __ffsll(u.Ny) - 1, ix, iy, iz);
  C cf[COEF_COUNT];
  constexpr int ncf = VAR == 2 ? COEF_COUNT : COEF_PSI1;
#pragma unroll
  for (int k = 0; k < ncf; ++k) cf[k] = cast_c<C>(__ldg(u.coef.full + k * u.nmode + m));
  update_one<VAR>(u, m, ix, iy, iz, cf);
}

// One thread per entry (qx, qy, iz) of the compact tables: the coefficients are read once and
// applied to the one, two or four modes (+-kx, +-ky, kz) that share them (qx = 0 and Nx / 2 have no
// mirror along x, likewise along y).  REAL: the standard variant's real tables.
// register caps: FP32 standard and Galilean variants 64 (4 CTAs per SM, no spills: 0.147 -> 0.128
// ms on the laser-wakefield box), the averaged variant 128 (at 80 its larger tables spill and it
// runs slower); FP64 128, and 255 for the averaged variant
template <int VAR, class C, bool REAL>
__global__ void __launch_bounds__(256, sizeof(C) == 8 ? (VAR == 2 ? 2 : 4) : (VAR == 2 ? 1 : 2))
    update_quad_kernel(UpdArgs<C> u) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= u.coef.nq) return;
  const uint32_t nzh = (uint32_t)u.nzh, nqy = (uint32_t)u.coef.nqy;
  const uint32_t ee = (uint32_t)e;
  const uint32_t r = ee / nzh, iz = ee - r * nzh;
  const uint32_t qx = r / nqy, qy = r - qx * nqy;
  C cf[COEF_COUNT];
  constexpr int ncf = VAR == 2 ? COEF_COUNT : COEF_PSI1;
#pragma unroll
  for (int k = 0; k < ncf; ++k) {
    if (sizeof(C) == 8 && u.coef.q32) {  // FP32 form: the tables' FP32 copy (same rounded values)
      if (REAL) {
        cf[k].x = __ldg(u.coef.q32 + k * u.coef.nq + e);
        cf[k].y = 0;
      } else {
        const float2 v = __ldg(reinterpret_cast<const float2*>(u.coef.q32) + k * u.coef.nq + e);
        cf[k].x = v.x;
        cf[k].y = v.y;
      }
    } else if (REAL) {
      cf[k].x = (decltype(C().x))__ldg(u.coef.q + k * u.coef.nq + e);
      cf[k].y = 0;
    } else {
      cf[k] = cast_c<C>(__ldg(reinterpret_cast<const double2*>(u.coef.q) + k * u.coef.nq + e));
    }
  }
  const uint32_t Nx = (uint32_t)u.coef.nx, Ny = (uint32_t)u.coef.ny;
  const int nmx = (qx == 0 || 2 * qx == Nx) ? 1 : 2, nmy = (qy == 0 || 2 * qy == Ny) ? 1 : 2;
  for (int a = 0; a < nmx; ++a) {
    const uint32_t ix = a ? Nx - qx : qx;
    for (int b = 0; b < nmy; ++b) {
      const uint32_t iy = b ? Ny - qy : qy;
      const int64_t m = ((int64_t)ix * Ny + iy) * nzh + iz;
      update_one<VAR>(u, m, ix, iy, iz, cf);
    }
  }
}

// staggering of each component kind: 0..5 = Ex..Bz, 6..8 = Jx..Jz, 9 = rho
__host__ __device__ __forceinline__ int stag_mask(int kind) {
  switch (kind) {
    case 0: case 6: return 1;   // x
    case 1: case 7: return 2;   // y
    case 2: case 8: return 4;   // z
    case 3: return 2 | 4;       // Bx: y, z
    case 4: return 1 | 4;       // By: x, z
    case 5: return 1 | 2;       // Bz: x, y
    default: return 0;
  }
}

// Conjugate transpose of the update (reverse mode).  Per mode, with K v = [k] x v:
//   Ebar = TC* Ebar' - i TS* K Bbar',  Bbar = TC* Bbar' + i c^2 TS* K Ebar',
//   Jbar = i X1* K Bbar' + X4* Ebar',  rhobar^n = -i TX3* k.Ebar',  rhobar^{n+1} = i X2* k.Ebar'.
// EB holds the adjoint spectra (paper convention) in and Ebar, Bbar out; G receives the nodal
// DFTs of Jbar (times zeta, the transpose of the J centering), rhobar^n and rhobar^{n+1}, / Ncell.
struct AdjUpdArgs {
  double2* EB;
  double2* G;
  const double2* coef;
  const double* ks[3];
  const double* zt[3];
  int64_t Ny, nzh, nmode;
  double c2, gscale;
};

__global__ void __launch_bounds__(256) adjoint_update_kernel(AdjUpdArgs u) {
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= u.nmode) return;
  const int64_t nm = u.nmode;
  const int64_t iz = m % u.nzh, r = m / u.nzh;
  const int64_t iy = r % u.Ny, ix = r / u.Ny;
  const double k[3] = {u.ks[0][ix], u.ks[1][iy], u.ks[2][iz]};
  const double zx = u.zt[0][ix], zy = u.zt[1][iy], zz = u.zt[2][iz];
  double2 E[3], B[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    E[a] = u.EB[a * nm + m];
    B[a] = u.EB[(3 + a) * nm + m];
  }
  auto cross = [&](const double2* F, double2* o) {
    o[0] = csub(cscale(F[2], k[1]), cscale(F[1], k[2]));
    o[1] = csub(cscale(F[0], k[2]), cscale(F[2], k[0]));
    o[2] = csub(cscale(F[1], k[0]), cscale(F[0], k[1]));
  };
  double2 KE[3], KB[3];
  cross(E, KE);
  cross(B, KB);
  auto co = [&](int idx) { return cconj(__ldg(u.coef + idx * nm + m)); };
  const double2 TC = co(COEF_TC), TS = co(COEF_TS), X1 = co(COEF_X1), X2 = co(COEF_X2), TX3 = co(COEF_TX3),
                X4 = co(COEF_X4);
  const double2 kE = cadd(cadd(cscale(E[0], k[0]), cscale(E[1], k[1])), cscale(E[2], k[2]));
  const double s = u.gscale;
  const double zj[3] = {zx, zy, zz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double2 Eo = csub(cmul(TC, E[a]), cmuli(cmul(TS, KB[a])));
    const double2 Bo = cadd(cmul(TC, B[a]), cmuli(cscale(cmul(TS, KE[a]), u.c2)));
    const double2 Jo = cadd(cmuli(cmul(X1, KB[a])), cmul(X4, E[a]));
    u.EB[a * nm + m] = Eo;
    u.EB[(3 + a) * nm + m] = Bo;
    u.G[a * nm + m] = cscale(Jo, zj[a] * s);
  }
  u.G[3 * nm + m] = cscale(cmuli(cmul(TX3, kE)), -s);
  u.G[4 * nm + m] = cscale(cmuli(cmul(X2, kE)), s);
}

// EB[c] += zeta_c * src[c]: adds the transpose of the E, B -> nodal centering (nodal DFTs in src).
struct AddZetaArgs {
  double2* EB;
  const double2* src;
  const double* zt[3];
  int64_t Ny, nzh, nmode;
};

__global__ void add_zeta_kernel(AddZetaArgs a) {
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= a.nmode) return;
  const int c = blockIdx.y;
  const int64_t iz = m % a.nzh, r = m / a.nzh;
  const int64_t iy = r % a.Ny, ix = r / a.Ny;
  const int mk = stag_mask(c);
  double z = 1.0;
  if (mk & 1) z *= a.zt[0][ix];
  if (mk & 2) z *= a.zt[1][iy];
  if (mk & 4) z *= a.zt[2][iz];
  a.EB[c * a.nmode + m] = cadd(a.EB[c * a.nmode + m], cscale(a.src[c * a.nmode + m], z));
}

template <class C>
struct PhaseArgs {
  CP6<C> in, out;
  int mask[6];
  int sign;
  double scale;
  const C* hs[3];  // half-cell shifts in the data precision
  int64_t Ny, nzh, nmode;
};

// The phase factors are formed in the data precision from 1D tables in that precision (GB300's FP64
// rate is a small fraction of its FP32 rate; in the FP32 form a product of up to three unit phases
// in FP32 is accurate to a few 1e-7, far below the transforms' own rounding).
template <class C>
__global__ void phase_kernel(PhaseArgs<C> p) {
  using T = decltype(C().x);
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= p.nmode) return;
  const int c = blockIdx.y;
  uint32_t ix, iy, iz;
  mode_xyz(m, (uint32_t)p.nzh, __ffsll(p.Ny) - 1, ix, iy, iz);
  C f;
  f.x = (T)p.scale;
  f.y = (T)0;
  const int mk = p.mask[c];
  if (mk & 1) f = cmul(f, p.hs[0][ix]);
  if (mk & 2) f = cmul(f, p.hs[1][iy]);
  if (mk & 4) f = cmul(f, p.hs[2][iz]);
  if (p.sign > 0) f.y = -f.y;
  p.out.p[c][m] = cmul(p.in.p[c][m], f);
}

template <class C>
struct NodalArgs {
  const C* EB;
  C* G;
  const decltype(C().x)* zt[3];  // centering symbols in the data precision
  int64_t Ny, nzh, nmode;
  double scale;
};

template <class C>
__global__ void to_nodal_kernel(NodalArgs<C> a) {
  using T = decltype(C().x);
  const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (m >= a.nmode) return;
  const int c = blockIdx.y;
  uint32_t ix, iy, iz;
  mode_xyz(m, (uint32_t)a.nzh, __ffsll(a.Ny) - 1, ix, iy, iz);
  const int mk = stag_mask(c);
  T z = (T)a.scale;
  if (mk & 1) z *= (T)a.zt[0][ix];
  if (mk & 2) z *= (T)a.zt[1][iy];
  if (mk & 4) z *= (T)a.zt[2][iz];
  a.G[c * a.nmode + m] = cscale(a.EB[c * a.nmode + m], z);
}

// ---------------------------------------------------------------------------
// host-side table construction (1D, exact rationals are not needed at FP64)
// ---------------------------------------------------------------------------
long double factl(int n) {
  long double f = 1.0L;
  for (int i = 2; i <= n; ++i) f *= (long double)i;
  return f;
}
// alpha^s_{m,n} (Eq. eq_Fornberg_staggered)
long double alpha_s(int m, int n) {
  long double dfact = 1.0L;  // (2m)! / (2^{2m} m!) = prod_{i=1}^m (2i-1)/2
  for (int i = 1; i <= m; ++i) dfact *= (2.0L * i - 1.0L) / 2.0L;
  const long double sgn = (n % 2 == 1) ? 1.0L : -1.0L;
  return sgn * dfact * dfact * 4.0L / ((2.0L * n - 1.0L) * factl(m - n) * factl(m + n - 1));
}
// alpha^c_{m,n} (Eq. eq_Fornberg_centered)
long double alpha_c(int m, int n) {
  const long double sgn = (n % 2 == 1) ? 1.0L : -1.0L;
  return sgn * 2.0L * factl(m) * factl(m) / (factl(m - n) * factl(m + n));
}

void gauss_legendre(GaussLegendre* g) {
  // Newton iteration on P_n in long double; nodes mapped to [0, 1], weights halved.
  const int n = kGL;
  const long double pi = 3.14159265358979323846264338327950288L;
  for (int i = 0; i < n; ++i) {
    long double x = cosl(pi * (i + 0.75L) / (n + 0.5L));
    long double dp = 0.0L;
    for (int it = 0; it < 100; ++it) {
      long double p0 = 1.0L, p1 = x;
      for (int k = 2; k <= n; ++k) {
        const long double p2 = ((2.0L * k - 1.0L) * x * p1 - (k - 1.0L) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (x * p1 - p0) / (x * x - 1.0L);
      const long double dx = p1 / dp;
      x -= dx;
      if (fabsl(dx) < 1e-30L) break;
    }
    {
      long double p0 = 1.0L, p1 = x;
      for (int k = 2; k <= n; ++k) {
        const long double p2 = ((2.0L * k - 1.0L) * x * p1 - (k - 1.0L) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (x * p1 - p0) / (x * x - 1.0L);
    }
    const long double w = 2.0L / ((1.0L - x * x) * dp * dp);
    g->x[i] = (double)(0.5L * (1.0L - x));
    g->w[i] = (double)(0.5L * w);
  }
}

}  // namespace

long double fornberg_alpha_s(int m, int n) { return alpha_s(m, n); }

pic_status psatd_setup(pic_ctx* ctx) {
  int64_t Nmax = std::max(ctx->N[0], std::max(ctx->N[1], ctx->N[2]));
  std::vector<double> h(9 * Nmax, 0.0);
  std::vector<double2> hs(3 * Nmax);
  for (int a = 0; a < 3; ++a) {
    const int64_t N = ctx->N[a];
    const double dx = ctx->dx[a];
    // FDTD cycle: ks is the symbol of its finite difference (order 2 when the order is 0)
    const int so = (ctx->cycle == PIC_CYCLE_HYBRID_FDTD && ctx->sorder[a] == 0) ? 2 : ctx->sorder[a];
    const int ms = so / 2, mc = ctx->corder[a] / 2;
    for (int64_t j = 0; j < N; ++j) {
      const int64_t js = j < N / 2 ? j : j - N;  // signed index, Nyquist -> -N/2
      double ks, kc, zeta = 0.0;
      if (ms == 0) {
        ks = kc = (double)(2.0L * 3.14159265358979323846264338327950288L * (long double)js / ((long double)N * dx));
      } else {
        long double sks = 0.0L, skc = 0.0L;
        for (int n = 1; n <= ms; ++n) {
          double s, c;
          sincospi_frac(js * (2 * n - 1), N, &s, &c);  // sin(k (n - 1/2) dx)
          sks += alpha_s(ms, n) * (long double)s / ((n - 0.5L) * dx);
          sincospi_frac(2 * js * n, N, &s, &c);        // sin(k n dx)
          skc += alpha_c(ms, n) * (long double)s / ((long double)n * dx);
        }
        ks = (double)sks;
        kc = (double)skc;
      }
      long double sz = 0.0L;
      for (int n = 1; n <= mc; ++n) {
        double s, c;
        sincospi_frac(js * (2 * n - 1), N, &s, &c);  // cos(k (n - 1/2) dx)
        sz += alpha_s(mc, n) * (long double)c;
      }
      zeta = (double)sz;
      double s, c;
      sincospi_frac(js, N, &s, &c);  // k dx / 2 = pi js / N
      double2 shift = make_double2(c, -s);
      if (ctx->cycle == PIC_CYCLE_NODAL) {
        // nodal comparison cycle (Sec. 2): node-based fields, [k]_c in the solver (0 at the
        // Nyquist index at infinite order: the centered derivative of node-based data), no
        // centering and no half-cell offsets
        if (ms == 0 && 2 * js == -N) kc = 0.0;
        ks = kc;
        zeta = 1.0;
        shift = make_double2(1.0, 0.0);
      }
      if (ctx->cycle == PIC_CYCLE_STAGGERED) zeta = 1.0;  // no centering in the staggered cycle
      h[(0 + a) * Nmax + j] = ks;
      h[(3 + a) * Nmax + j] = kc;
      h[(6 + a) * Nmax + j] = zeta;
      hs[a * Nmax + j] = shift;
    }
    ctx->cw[a].m = mc;
    for (int n = 1; n <= mc; ++n) ctx->cw[a].w[n - 1] = (double)(alpha_s(mc, n) / 2.0L);
  }
  PIC_CUDA_TRY(ctx, cudaMalloc(&ctx->k1d, 9 * Nmax * sizeof(double) + 3 * Nmax * sizeof(double2)));
  PIC_CUDA_TRY(ctx, cudaMemcpy(ctx->k1d, h.data(), 9 * Nmax * sizeof(double), cudaMemcpyHostToDevice));
  double2* hsd = reinterpret_cast<double2*>(ctx->k1d + 9 * Nmax);
  PIC_CUDA_TRY(ctx, cudaMemcpy(hsd, hs.data(), 3 * Nmax * sizeof(double2), cudaMemcpyHostToDevice));
  for (int a = 0; a < 3; ++a) {
    ctx->ks[a] = ctx->k1d + (0 + a) * Nmax;
    ctx->kc[a] = ctx->k1d + (3 + a) * Nmax;
    ctx->zeta[a] = ctx->k1d + (6 + a) * Nmax;
  }
  {
    // FP32 copies of the same 1D tables (same layout), rounded once here
    std::vector<float> h32(9 * Nmax + 6 * Nmax);
    for (int64_t i = 0; i < 9 * Nmax; ++i) h32[i] = (float)h[i];
    for (int64_t i = 0; i < 3 * Nmax; ++i) {
      h32[9 * Nmax + 2 * i] = (float)hs[i].x;
      h32[9 * Nmax + 2 * i + 1] = (float)hs[i].y;
    }
    PIC_CUDA_TRY(ctx, cudaMalloc(&ctx->k1d32, h32.size() * sizeof(float)));
    PIC_CUDA_TRY(ctx, cudaMemcpy(ctx->k1d32, h32.data(), h32.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  // bilinear filter symbols (Sec. 2): per pass and axis, (1/4, 1/2, 1/4) -> cos^2(k dx / 2)
  if (ctx->filter_passes > 0) {
    std::vector<double> hf(3 * Nmax, 0.0);
    for (int a = 0; a < 3; ++a) {
      const int64_t N = ctx->N[a];
      for (int64_t j = 0; j < N; ++j) {
        const int64_t js = j < N / 2 ? j : j - N;
        double s, c;
        sincospi_frac(js, N, &s, &c);  // cos(k dx / 2)
        double f = 1.0;
        for (int q = 0; q < ctx->filter_passes; ++q) f *= c * c;
        hf[a * Nmax + j] = f;
      }
    }
    PIC_CUDA_TRY(ctx, cudaMalloc(&ctx->flt1d, 3 * Nmax * sizeof(double)));
    PIC_CUDA_TRY(ctx, cudaMemcpy(ctx->flt1d, hf.data(), 3 * Nmax * sizeof(double), cudaMemcpyHostToDevice));
    for (int a = 0; a < 3; ++a) ctx->flt[a] = ctx->flt1d + a * Nmax;
    std::vector<float> hf32(hf.begin(), hf.end());
    PIC_CUDA_TRY(ctx, cudaMalloc(&ctx->flt32, 3 * Nmax * sizeof(float)));
    PIC_CUDA_TRY(ctx, cudaMemcpy(ctx->flt32, hf32.data(), 3 * Nmax * sizeof(float), cudaMemcpyHostToDevice));
  }
  // keep the half-cell shift tables right after the 1D tables
  ctx->ncoef = ctx->variant == PIC_PSATD_AVERAGED_GALILEAN ? COEF_COUNT : COEF_PSI1;
  PIC_CUDA_TRY(ctx, cudaMalloc(&ctx->coef, (size_t)ctx->ncoef * ctx->nmode * sizeof(double2)));
  TableArgs t;
  for (int a = 0; a < 3; ++a) {
    t.ks[a] = ctx->ks[a];
    t.kc[a] = ctx->kc[a];
    t.vg[a] = ctx->variant == PIC_PSATD_STANDARD ? 0.0 : ctx->vg[a];
  }
  t.Ny = ctx->N[1];
  t.nzh = ctx->nzh;
  t.nmode = ctx->nmode;
  t.dt = ctx->dt;
  t.c = ctx->c;
  t.eps0 = ctx->eps0;
  t.ncoef = ctx->ncoef;
  t.averaged = ctx->variant == PIC_PSATD_AVERAGED_GALILEAN;
  t.coef = ctx->coef;
  gauss_legendre(&t.gl);
  const int bs = 128;
  build_tables_kernel<<<(unsigned)((ctx->nmode + bs - 1) / bs), bs, 0, ctx->stream>>>(t);
  PIC_LAUNCH_CHECK(ctx);
  // compact tables for the step's update (see pic_ctx::coefq)
  ctx->coefq = nullptr;
  ctx->coefq32 = nullptr;
  if (ctx->variant == PIC_PSATD_STANDARD || (ctx->vg[0] == 0.0 && ctx->vg[1] == 0.0)) {
    ctx->coefq_real = ctx->variant == PIC_PSATD_STANDARD ? 1 : 0;
    ctx->nqx = ctx->N[0] / 2 + 1;
    ctx->nqy = ctx->N[1] / 2 + 1;
    ctx->nq = ctx->nqx * ctx->nqy * ctx->nzh;
    const size_t words = (size_t)ctx->ncoef * ctx->nq * (ctx->coefq_real ? 1 : 2);
    PIC_CUDA_TRY(ctx, cudaMalloc(&ctx->coefq, words * sizeof(double)));
    if (ctx->precision == PIC_FP32) PIC_CUDA_TRY(ctx, cudaMalloc(&ctx->coefq32, words * sizeof(float)));
    CompactArgs c;
    c.full = ctx->coef;
    c.q = ctx->coefq;
    c.q32 = ctx->coefq32;
    c.real = ctx->coefq_real;
    c.ncoef = ctx->ncoef;
    c.Ny = ctx->N[1];
    c.nzh = ctx->nzh;
    c.nqy = ctx->nqy;
    c.nq = ctx->nq;
    c.nmode = ctx->nmode;
    compact_tables_kernel<<<(unsigned)((ctx->nq + 255) / 256), 256, 0, ctx->stream>>>(c);
    PIC_LAUNCH_CHECK(ctx);
  }
  PIC_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return PIC_OK;
}

static const double2* half_shift(const pic_ctx* ctx, int a) {
  const int64_t Nmax = std::max(ctx->N[0], std::max(ctx->N[1], ctx->N[2]));
  return reinterpret_cast<const double2*>(ctx->k1d + 9 * Nmax) + a * Nmax;
}

// 1D tables of axis a ([k]_s, zeta, filter symbols or NULL, half-cell shifts) in FP64 or FP32
static void tab1d(const pic_ctx* ctx, int a, const double** ks, const double** zt, const double** flt,
                  const double2** hs) {
  *ks = ctx->ks[a];
  *zt = ctx->zeta[a];
  *flt = ctx->filter_passes > 0 ? ctx->flt[a] : nullptr;
  *hs = half_shift(ctx, a);
}
static void tab1d(const pic_ctx* ctx, int a, const float** ks, const float** zt, const float** flt,
                  const float2** hs) {
  const int64_t Nmax = std::max(ctx->N[0], std::max(ctx->N[1], ctx->N[2]));
  *ks = ctx->k1d32 + (0 + a) * Nmax;
  *zt = ctx->k1d32 + (6 + a) * Nmax;
  *flt = ctx->filter_passes > 0 ? ctx->flt32 + a * Nmax : nullptr;
  *hs = reinterpret_cast<const float2*>(ctx->k1d32 + 9 * Nmax) + a * Nmax;
}

template <class C>
pic_status psatd_update_t(pic_ctx* ctx, C* EB, C* J, const C* rn, const C* rp, C* G, int g_mode, int j_yee,
                          int write_j, int smooth) {
  UpdArgs<C> u;
  u.EB = EB;
  u.J = J;
  u.rn = rn;
  u.rp = rp;
  u.coef = coef_view(ctx);
  u.G = G;
  for (int a = 0; a < 3; ++a) {
    tab1d(ctx, a, &u.ks[a], &u.zt[a], &u.flt[a], &u.hs[a]);
    if (!(smooth && ctx->filter_passes > 0)) u.flt[a] = nullptr;
  }
  u.Ny = ctx->N[1];
  u.nzh = ctx->nzh;
  u.nmode = ctx->nmode;
  u.c2 = ctx->c * ctx->c;
  u.gscale = 1.0 / (double)ctx->ncell;
  u.g_mode = g_mode;
  u.j_yee = j_yee;
  u.write_j = write_j;
  const int bs = 256;
  const bool avg = ctx->variant == PIC_PSATD_AVERAGED_GALILEAN;
  if (ctx->coefq) {
    const unsigned nb = (unsigned)((ctx->nq + bs - 1) / bs);
    if (avg) update_quad_kernel<2, C, false><<<nb, bs, 0, ctx->stream>>>(u);
    else if (ctx->coefq_real) update_quad_kernel<0, C, true><<<nb, bs, 0, ctx->stream>>>(u);
    else update_quad_kernel<0, C, false><<<nb, bs, 0, ctx->stream>>>(u);
  } else {
    const unsigned nb = (unsigned)((ctx->nmode + bs - 1) / bs);
    if (avg) update_kernel<2, C><<<nb, bs, 0, ctx->stream>>>(u);
    else update_kernel<0, C><<<nb, bs, 0, ctx->stream>>>(u);
  }
  PIC_LAUNCH_CHECK(ctx);
  return PIC_OK;
}

pic_status psatd_update_ex(pic_ctx* ctx, const double2* rn, const double2* rp, int g_mode, int j_yee,
                           int write_j, int smooth) {
  return psatd_update_t<double2>(ctx, ctx->EBh, ctx->Jh, rn, rp, ctx->G, g_mode, j_yee, write_j, smooth);
}

pic_status psatd_update32(pic_ctx* ctx, float2* EB, float2* J, const float2* rn, const float2* rp, float2* G,
                          int g_mode, int j_yee, int write_j, int smooth) {
  return psatd_update_t<float2>(ctx, EB, J, rn, rp, G, g_mode, j_yee, write_j, smooth);
}

pic_status psatd_update(pic_ctx* ctx, int cur) {
  return psatd_update_ex(ctx, ctx->rhoh[cur], ctx->rhoh[1 - cur], 0, 0, 1, 1);
}

template <class C>
pic_status psatd_phase_t(pic_ctx* ctx, CP6<C> in, CP6<C> out, const int* comp_kind, int ncomp, int sign,
                         double scale) {
  PhaseArgs<C> p;
  p.in = in;
  p.out = out;
  for (int c = 0; c < ncomp; ++c) p.mask[c] = stag_mask(comp_kind[c]);
  p.sign = sign;
  p.scale = scale;
  for (int a = 0; a < 3; ++a) {
    const C* h;
    const decltype(C().x)* unused[3];
    tab1d(ctx, a, &unused[0], &unused[1], &unused[2], &h);
    p.hs[a] = h;
  }
  p.Ny = ctx->N[1];
  p.nzh = ctx->nzh;
  p.nmode = ctx->nmode;
  const int bs = 256;
  dim3 grid((unsigned)((ctx->nmode + bs - 1) / bs), ncomp);
  phase_kernel<C><<<grid, bs, 0, ctx->stream>>>(p);
  PIC_LAUNCH_CHECK(ctx);
  return PIC_OK;
}

pic_status psatd_phase(pic_ctx* ctx, CPtr6 in, CPtr6 out, const int* comp_kind, int ncomp, int sign,
                       double scale) {
  return psatd_phase_t<double2>(ctx, in, out, comp_kind, ncomp, sign, scale);
}

pic_status psatd_phase32(pic_ctx* ctx, CP6<float2> in, CP6<float2> out, const int* comp_kind, int ncomp, int sign,
                         double scale) {
  return psatd_phase_t<float2>(ctx, in, out, comp_kind, ncomp, sign, scale);
}

template <class C>
pic_status psatd_to_nodal_t(pic_ctx* ctx, const C* EB6, C* G, double scale) {
  NodalArgs<C> a;
  a.EB = EB6;
  a.G = G;
  for (int k = 0; k < 3; ++k) {
    const decltype(C().x)* unused[2];
    const C* h;
    tab1d(ctx, k, &unused[0], &a.zt[k], &unused[1], &h);
  }
  a.Ny = ctx->N[1];
  a.nzh = ctx->nzh;
  a.nmode = ctx->nmode;
  a.scale = scale;
  const int bs = 256;
  dim3 grid((unsigned)((ctx->nmode + bs - 1) / bs), 6);
  to_nodal_kernel<C><<<grid, bs, 0, ctx->stream>>>(a);
  PIC_LAUNCH_CHECK(ctx);
  return PIC_OK;
}

pic_status psatd_to_nodal(pic_ctx* ctx, const double2* EB6, double scale) {
  return psatd_to_nodal_t<double2>(ctx, EB6, ctx->G, scale);
}

pic_status psatd_to_nodal32(pic_ctx* ctx, const float2* EB6, float2* G, double scale) {
  return psatd_to_nodal_t<float2>(ctx, EB6, G, scale);
}

pic_status psatd_adjoint_update(pic_ctx* ctx, double2* EB, double2* G) {
  AdjUpdArgs u;
  u.EB = EB;
  u.G = G;
  u.coef = ctx->coef;
  for (int a = 0; a < 3; ++a) {
    u.ks[a] = ctx->ks[a];
    u.zt[a] = ctx->zeta[a];
  }
  u.Ny = ctx->N[1];
  u.nzh = ctx->nzh;
  u.nmode = ctx->nmode;
  u.c2 = ctx->c * ctx->c;
  u.gscale = 1.0 / (double)ctx->ncell;
  const int bs = 256;
  adjoint_update_kernel<<<(unsigned)((ctx->nmode + bs - 1) / bs), bs, 0, ctx->stream>>>(u);
  PIC_LAUNCH_CHECK(ctx);
  return PIC_OK;
}

pic_status psatd_add_zeta(pic_ctx* ctx, double2* EB, const double2* src) {
  AddZetaArgs a;
  a.EB = EB;
  a.src = src;
  for (int k = 0; k < 3; ++k) a.zt[k] = ctx->zeta[k];
  a.Ny = ctx->N[1];
  a.nzh = ctx->nzh;
  a.nmode = ctx->nmode;
  const int bs = 256;
  dim3 grid((unsigned)((ctx->nmode + bs - 1) / bs), 6);
  add_zeta_kernel<<<grid, bs, 0, ctx->stream>>>(a);
  PIC_LAUNCH_CHECK(ctx);
  return PIC_OK;
}
