// 3D real-to-complex FFT for the PSATD solver: shared-memory Stockham kernels.
//
// Forward: z-axis R2C (a length-Nz/2 complex FFT of packed (even, odd) pairs
// followed by the split step), then in-place C2C along y and along x.
// Inverse: C2C along x, along y, then z-axis C2R.  Plain DFT, unnormalised:
// X_m = sum_j x_j exp(-2 pi i j.m / N) (App. A.1, Eq. Fourier_discrete without
// the half-cell phase, which the caller applies).
//
// Every CTA loads a whole tile of lines into shared memory, runs the radix-8
// (+ one radix-4 or radix-2) Stockham passes there, and writes the tile back.
// z lines are contiguous (line-major tile, padded one slot per 8 elements to
// keep the radix-8 scatter conflict-free); y and x lines are strided, so a CTA
// takes W adjacent columns (consecutive k_z) and the tile is element-major,
// which keeps the global loads coalesced in W * 16-byte rows.
#include "pic_internal.cuh"

#include <cmath>

namespace {

constexpr int kZTile = 4096;    // complex elements per z-pass CTA (L lines * Nz/2)
constexpr int kMaxThreads = 1024;

struct LayLine {  // z pass: element e of line l at l * LP + e + e / 8
  int LP;
  __device__ __forceinline__ int idx(int e, int l) const { return l * LP + e + (e >> 3); }
  __device__ __forceinline__ void map(int b, int nb, int& l, int& j) const {
    l = b / nb;
    j = b - l * nb;
  }
};

struct LayCol {  // y / x pass: element e of column w at e * W + w
  int W;
  __device__ __forceinline__ int idx(int e, int w) const { return e * W + w; }
  __device__ __forceinline__ void map(int b, int nb, int& l, int& j) const {
    j = b / W;
    l = b - j * W;
  }
};

// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ double2 rot90(double2 a) {
  return INV ? make_double2(-a.y, a.x) : make_double2(a.y, -a.x);
}

template <bool INV>
__device__ __forceinline__ void dft4(double2& y0, double2& y1, double2& y2, double2& y3) {
  double2 t0 = cadd(y0, y2), t1 = csub(y0, y2);
  double2 t2 = cadd(y1, y3), t3 = rot90<INV>(csub(y1, y3));
  y0 = cadd(t0, t2);
  y2 = csub(t0, t2);
  y1 = cadd(t1, t3);
  y3 = csub(t1, t3);
}

template <int R, bool INV>
__device__ __forceinline__ void dft(double2* v) {
  if (R == 2) {
    double2 a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
  } else if (R == 4) {
    dft4<INV>(v[0], v[1], v[2], v[3]);
  } else {  // R == 8: radix-2 split over n and n+4, then two radix-4 DFTs
    const double r2 = 0.70710678118654752440;
    double2 b[4], c[4];
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      b[n] = cadd(v[n], v[n + 4]);
      c[n] = csub(v[n], v[n + 4]);
    }
    // c_n *= w8^n, w8 = exp(-+ 2 pi i / 8)
    if (INV) {
      c[1] = make_double2((c[1].x - c[1].y) * r2, (c[1].x + c[1].y) * r2);
      c[3] = make_double2((-c[3].x - c[3].y) * r2, (c[3].x - c[3].y) * r2);
    } else {
      c[1] = make_double2((c[1].x + c[1].y) * r2, (c[1].y - c[1].x) * r2);
      c[3] = make_double2((c[3].y - c[3].x) * r2, (-c[3].x - c[3].y) * r2);
    }
    c[2] = rot90<INV>(c[2]);
    dft4<INV>(b[0], b[1], b[2], b[3]);
    dft4<INV>(c[0], c[1], c[2], c[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[2 * k] = b[k];
      v[2 * k + 1] = c[k];
    }
  }
}

// One Stockham pass of radix R on all lines of the tile, in place.  The CTA has
// exactly L * N / 8 threads; each thread handles 8 / R butterflies.
template <int R, bool INV, class LAY>
__device__ __forceinline__ void stockham_pass(double2* s, const LAY& lay, int N, int Ns,
                                              const double2* __restrict__ tw, int twstride) {
  constexpr int PER = 8 / R;
  const int T = blockDim.x;
  const int nb = N / R;
  double2 v[PER][R];
  int ol[PER], oj[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    int b = threadIdx.x + q * T;
    int l, j;
    lay.map(b, nb, l, j);
    ol[q] = l;
    oj[q] = j;
#pragma unroll
    for (int r = 0; r < R; ++r) v[q][r] = s[lay.idx(j + r * nb, l)];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int j = oj[q], l = ol[q];
    const int k = j & (Ns - 1);
    if (Ns > 1) {
      const int step = (N / (Ns * R)) * k;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        double2 w = __ldg(&tw[step * r * twstride]);
        if (INV) w.y = -w.y;
        v[q][r] = cmul(v[q][r], w);
      }
    }
    dft<R, INV>(v[q]);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) s[lay.idx(base + r * Ns, l)] = v[q][r];
  }
  __syncthreads();
}

template <bool INV, class LAY>
__device__ void fft_tile(double2* s, const LAY& lay, int N, const double2* __restrict__ tw, int twstride) {
  int Ns = 1, rem = N;
  while (rem >= 8) {
    stockham_pass<8, INV>(s, lay, N, Ns, tw, twstride);
    Ns *= 8;
    rem /= 8;
  }
  if (rem == 4) stockham_pass<4, INV>(s, lay, N, Ns, tw, twstride);
  else if (rem == 2) stockham_pass<2, INV>(s, lay, N, Ns, tw, twstride);
}

// z-axis real-to-complex: L lines of Nz reals -> Nz/2+1 complex per line.
__global__ void __launch_bounds__(kMaxThreads) fft_z_r2c_kernel(CRPtr6 in, CPtr6 out, int Nz, int64_t nlines,
                                                               int L, const double2* __restrict__ tw) {
  extern __shared__ double2 sm[];
  const int M = Nz / 2;
  const LayLine lay{M + M / 8};
  const int comp = blockIdx.y;
  const int64_t line0 = (int64_t)blockIdx.x * L;
  const double2* src = reinterpret_cast<const double2*>(in.p[comp]);
  for (int t = threadIdx.x; t < L * M; t += blockDim.x) {
    const int l = t / M, e = t - l * M;
    const int64_t line = line0 + l;
    sm[lay.idx(e, l)] = line < nlines ? src[line * M + e] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  fft_tile<false>(sm, lay, M, tw, 2);
  // split: X_k = (Z_k + conj Z_{M-k})/2 - (i/2) W^k (Z_k - conj Z_{M-k}),  W = exp(-2 pi i / Nz)
  double2* dst = out.p[comp];
  const int nzh = M + 1, P = M / 2 + 1;
  for (int t = threadIdx.x; t < L * P; t += blockDim.x) {
    const int l = t / P, k = t - l * P;
    const int64_t line = line0 + l;
    if (line >= nlines) continue;
    const double2 Zk = sm[lay.idx(k, l)];
    const double2 Zm = sm[lay.idx((M - k) & (M - 1), l)];
    const double2 Fe = make_double2(0.5 * (Zk.x + Zm.x), 0.5 * (Zk.y - Zm.y));
    const double2 Fo = make_double2(0.5 * (Zk.y + Zm.y), -0.5 * (Zk.x - Zm.x));
    const double2 wFo = cmul(__ldg(&tw[k]), Fo);
    double2* o = dst + line * nzh;
    o[k] = cadd(Fe, wFo);
    if (k != M - k) o[M - k] = cconj(csub(Fe, wFo));
  }
}

// z-axis complex-to-real (unnormalised inverse); the imaginary parts of X_0, X_{Nz/2} are ignored.
__global__ void __launch_bounds__(kMaxThreads) fft_z_c2r_kernel(CPtr6 in, RPtr6 out, int Nz, int64_t nlines,
                                                               int L, const double2* __restrict__ tw) {
  extern __shared__ double2 sm[];
  const int M = Nz / 2;
  const LayLine lay{M + M / 8};
  const int comp = blockIdx.y;
  const int64_t line0 = (int64_t)blockIdx.x * L;
  const double2* srcb = in.p[comp];
  const int nzh = M + 1, P = M / 2 + 1;
  // Z_k = (X_k + conj X_{M-k}) + i W^{-k} (X_k - conj X_{M-k})
  for (int t = threadIdx.x; t < L * P; t += blockDim.x) {
    const int l = t / P, k = t - l * P;
    const int64_t line = line0 + l;
    double2 Xk = make_double2(0.0, 0.0), Xm = make_double2(0.0, 0.0);
    if (line < nlines) {
      Xk = srcb[line * nzh + k];
      Xm = srcb[line * nzh + (M - k)];
    }
    if (k == 0) {
      Xk.y = 0.0;
      Xm.y = 0.0;
    }
    const double2 A = make_double2(Xk.x + Xm.x, Xk.y - Xm.y);
    const double2 D = make_double2(Xk.x - Xm.x, Xk.y + Xm.y);
    const double2 w = __ldg(&tw[k]);
    sm[lay.idx(k, l)] = cadd(A, cmuli(cmul(cconj(w), D)));
    if (k != 0 && k != M - k) sm[lay.idx(M - k, l)] = cadd(cconj(A), cmuli(cmul(w, cconj(D))));
  }
  __syncthreads();
  fft_tile<true>(sm, lay, M, tw, 2);
  double2* dst = reinterpret_cast<double2*>(out.p[comp]);
  for (int t = threadIdx.x; t < L * M; t += blockDim.x) {
    const int l = t / M, e = t - l * M;
    const int64_t line = line0 + l;
    if (line < nlines) dst[line * M + e] = sm[lay.idx(e, l)];
  }
}

// In-place C2C along a strided axis: element e of column col of outer line o of
// component c at p[c] + o * os + e * es + col.  A CTA takes W adjacent columns.
template <bool INV>
__global__ void __launch_bounds__(kMaxThreads) fft_strided_kernel(CPtr6 data, int N, int64_t es, int64_t os,
                                                                 int ncols, int W, const double2* __restrict__ tw) {
  extern __shared__ double2 sm[];
  const LayCol lay{W};
  const int comp = blockIdx.z;
  const int col0 = blockIdx.x * W;
  double2* base = data.p[comp] + (int64_t)blockIdx.y * os + col0;
  const int wv = min(W, ncols - col0);
  for (int t = threadIdx.x; t < N * W; t += blockDim.x) {
    const int e = t / W, w = t - e * W;
    sm[t] = w < wv ? base[e * es + w] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  fft_tile<INV>(sm, lay, N, tw, 1);
  for (int t = threadIdx.x; t < N * W; t += blockDim.x) {
    const int e = t / W, w = t - e * W;
    if (w < wv) base[e * es + w] = sm[t];
  }
}

int strided_width(int N) { return N >= 1024 ? 8 : 16; }

pic_status launch_strided(pic_ctx* ctx, CPtr6 d, int axis, bool inv, int ncomp) {
  const int N = (int)ctx->N[axis];
  const int W = strided_width(N);
  const int nzh = (int)ctx->nzh;
  int64_t es, os, nouter;
  if (axis == 1) {  // y: outer = x
    es = nzh;
    os = ctx->N[1] * nzh;
    nouter = ctx->N[0];
  } else {  // x: outer = y
    es = ctx->N[1] * nzh;
    os = nzh;
    nouter = ctx->N[1];
  }
  dim3 grid((nzh + W - 1) / W, (unsigned)nouter, ncomp);
  const int threads = W * N / 8;
  const size_t smem = (size_t)W * N * sizeof(double2);
  if (inv)
    fft_strided_kernel<true><<<grid, threads, smem, ctx->stream>>>(d, N, es, os, nzh, W, ctx->twid[axis]);
  else
    fft_strided_kernel<false><<<grid, threads, smem, ctx->stream>>>(d, N, es, os, nzh, W, ctx->twid[axis]);
  PIC_LAUNCH_CHECK(ctx);
  return PIC_OK;
}

int z_lines_per_cta(int Nz) { return kZTile / (Nz / 2); }

}  // namespace

void sincospi_frac(int64_t p, int64_t q, double* s, double* c) {
  // sin, cos of pi p / q with the angle reduced on integers; exact at multiples of pi/2.
  int64_t r = p % (2 * q);
  if (r < 0) r += 2 * q;
  if ((2 * r) % q == 0) {
    const int64_t quarter = (2 * r) / q;  // 0..3
    const double sv[4] = {0.0, 1.0, 0.0, -1.0}, cv[4] = {1.0, 0.0, -1.0, 0.0};
    *s = sv[quarter];
    *c = cv[quarter];
    return;
  }
  const long double pi = 3.14159265358979323846264338327950288L;
  const long double a = pi * (long double)r / (long double)q;
  *s = (double)sinl(a);
  *c = (double)cosl(a);
}

pic_status fft_setup(pic_ctx* ctx) {
  for (int a = 0; a < 3; ++a) {
    const int64_t N = ctx->N[a];
    double2* h = new double2[N];
    for (int64_t j = 0; j < N; ++j) {
      double s, c;
      sincospi_frac(2 * j, N, &s, &c);
      h[j] = make_double2(c, -s);  // exp(-2 pi i j / N)
    }
    cudaError_t e = cudaMalloc(&ctx->twid[a], N * sizeof(double2));
    if (e == cudaSuccess) e = cudaMemcpy(ctx->twid[a], h, N * sizeof(double2), cudaMemcpyHostToDevice);
    delete[] h;
    if (e != cudaSuccess) return pic_set_error(ctx, PIC_ERR_NOMEM, "twiddle table: %s", cudaGetErrorString(e));
  }
  const int zsm = kZTile * 9 / 8 * (int)sizeof(double2);
  PIC_CUDA_TRY(ctx, cudaFuncSetAttribute(fft_z_r2c_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, zsm));
  PIC_CUDA_TRY(ctx, cudaFuncSetAttribute(fft_z_c2r_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, zsm));
  const int ssm = 8192 * (int)sizeof(double2);
  PIC_CUDA_TRY(ctx, cudaFuncSetAttribute(fft_strided_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, ssm));
  PIC_CUDA_TRY(ctx, cudaFuncSetAttribute(fft_strided_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ssm));
  return PIC_OK;
}

pic_status fft_r2c(pic_ctx* ctx, CRPtr6 in, CPtr6 out, int ncomp) {
  const int Nz = (int)ctx->N[2];
  const int L = z_lines_per_cta(Nz);
  const int64_t nlines = ctx->N[0] * ctx->N[1];
  dim3 grid((unsigned)((nlines + L - 1) / L), ncomp);
  const size_t smem = (size_t)L * (Nz / 2 + Nz / 16) * sizeof(double2);
  fft_z_r2c_kernel<<<grid, L * (Nz / 2) / 8, smem, ctx->stream>>>(in, out, Nz, nlines, L, ctx->twid[2]);
  PIC_LAUNCH_CHECK(ctx);
  pic_status st = launch_strided(ctx, out, 1, false, ncomp);
  if (st != PIC_OK) return st;
  return launch_strided(ctx, out, 0, false, ncomp);
}

pic_status fft_c2r(pic_ctx* ctx, CPtr6 in, RPtr6 out, int ncomp) {
  pic_status st = launch_strided(ctx, in, 0, true, ncomp);
  if (st != PIC_OK) return st;
  st = launch_strided(ctx, in, 1, true, ncomp);
  if (st != PIC_OK) return st;
  const int Nz = (int)ctx->N[2];
  const int L = z_lines_per_cta(Nz);
  const int64_t nlines = ctx->N[0] * ctx->N[1];
  dim3 grid((unsigned)((nlines + L - 1) / L), ncomp);
  const size_t smem = (size_t)L * (Nz / 2 + Nz / 16) * sizeof(double2);
  fft_z_c2r_kernel<<<grid, L * (Nz / 2) / 8, smem, ctx->stream>>>(in, out, Nz, nlines, L, ctx->twid[2]);
  PIC_LAUNCH_CHECK(ctx);
  return PIC_OK;
}
