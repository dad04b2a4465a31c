// 3D real-to-complex FFT for the PSATD solver: shared-memory Stockham kernels,
// templated on the precision (FP64 form: double; FP32 form: float).
//
// Forward: z-axis R2C (a length-Nz/2 complex FFT of packed (even, odd) pairs
// followed by the split step), then in-place C2C along y and along x.
// Inverse: C2C along x, along y, then z-axis C2R.  Plain DFT, unnormalised:
// X_m = sum_j x_j exp(-2 pi i j.m / N) (App. A.1, Eq. Fourier_discrete without
// the half-cell phase, which the caller applies).
//
// Every CTA transforms a whole tile of lines: radix-8 (+ one radix-4 or radix-2) Stockham passes
// with every length a template parameter (one kernel per power of two, all index arithmetic
// compile-time shifts and masks).  Pass 0 takes its butterfly's inputs straight from global memory
// into registers, the last pass of a C2C or C2R transform writes straight back, so a transform of
// npass passes goes through shared memory npass - 1 times.  z lines are contiguous (line-major
// tile, padded 2 slots per 16 elements to spread the radix-8 scatter over the banks); y and x
// lines are strided, so a CTA takes W adjacent columns (consecutive k_z) and the tile is
// element-major, which keeps the global loads coalesced in W-element rows.
#include "pic_internal.cuh"
#include "fft_tile.cuh"

#include <cmath>

namespace {

constexpr int kZTile = 4096;  // complex elements per z-pass CTA (L lines * Nz/2): 512 threads

using namespace pic_fft;

// z-axis real-to-complex: L = 4096 / M lines of Nz = 2M reals -> M + 1 complex per line.  Each
// thread loads its pass-0 butterfly (8 packed (even, odd) pairs, stride M / 8) straight from global
// memory.
template <class T, int LGM>
__global__ void __launch_bounds__(512, sizeof(T) == 4 ? 3 : 2)
    fft_z_r2c_kernel(CRP6<T> in, CP6<typename Cplx<T>::type> out, int64_t nlines,
                     const typename Cplx<T>::type* __restrict__ tw) {
  using C = typename Cplx<T>::type;
  constexpr int M = 1 << LGM, L = kZTile / M, lgnb = LGM - 3, nb = 1 << lgnb;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const LayLine lay{zline_len(M)};
  const int comp = blockIdx.y;
  const int64_t line0 = (int64_t)blockIdx.x * L;
  {
    const int l = threadIdx.x >> lgnb, j = threadIdx.x & (nb - 1);
    const int64_t line = line0 + l;
    const C* src = reinterpret_cast<const C*>(in.p[comp]) + line * M + j;
    C v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = line < nlines ? src[r * nb] : czero<C>();
    pass0_from_regs<false>(sm, lay, v, j, l);
  }
  passes_ct<false, LGM, 1, Plan<LGM>::npass>(sm, lay, tw, 2);
  // split: X_k = (Z_k + conj Z_{M-k})/2 - (i/2) W^k (Z_k - conj Z_{M-k}),  W = exp(-2 pi i / Nz)
  C* dst = out.p[comp];
  constexpr int nzh = M + 1, lgH = LGM - 1;
  const T h = (T)0.5;
  // k = 0 .. M/2 - 1 for every line (t < L M / 2), then k = M/2 (t >= L M / 2)
  for (int t = threadIdx.x; t < (L << lgH) + L; t += blockDim.x) {
    const bool mid = t >= (L << lgH);
    const int l = mid ? t - (L << lgH) : t >> lgH;
    const int k = mid ? (M >> 1) : t & ((M >> 1) - 1);
    const int64_t line = line0 + l;
    if (line >= nlines) continue;
    const C Zk = sm[lay.idx(k, l)];
    const C Zm = sm[lay.idx((M - k) & (M - 1), l)];
    C Fe, Fo;
    Fe.x = h * (Zk.x + Zm.x);
    Fe.y = h * (Zk.y - Zm.y);
    Fo.x = h * (Zk.y + Zm.y);
    Fo.y = -h * (Zk.x - Zm.x);
    const C wFo = cmul(__ldg(&tw[k]), Fo);
    C* o = dst + line * nzh;
    o[k] = cadd(Fe, wFo);
    if (k != M - k) o[M - k] = cconj(csub(Fe, wFo));
  }
}

// z-axis complex-to-real (unnormalised inverse); the imaginary parts of X_0, X_{Nz/2} are ignored.
// The last pass writes its outputs straight to global memory.
template <class T, int LGM>
__global__ void __launch_bounds__(512, sizeof(T) == 4 ? 3 : 2)
    fft_z_c2r_kernel(CP6<typename Cplx<T>::type> in, RP6<T> out, int64_t nlines,
                     const typename Cplx<T>::type* __restrict__ tw) {
  using C = typename Cplx<T>::type;
  constexpr int M = 1 << LGM, L = kZTile / M;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const LayLine lay{zline_len(M)};
  const int comp = blockIdx.y;
  const int64_t line0 = (int64_t)blockIdx.x * L;
  const C* srcb = in.p[comp];
  constexpr int nzh = M + 1, P = M / 2 + 1, lgH = LGM - 1;
  // Z_k = (X_k + conj X_{M-k}) + i W^{-k} (X_k - conj X_{M-k})
  // k = 0 .. M/2 - 1 for every line (t < L M / 2), then k = M/2 (t >= L M / 2)
  constexpr int kBatch = (L * P + 511) / 512;  // L * P <= 5 * 512 for every M >= 8
  C xk[kBatch], xm[kBatch];
#pragma unroll
  for (int q = 0; q < kBatch; ++q) {
    const int t = threadIdx.x + q * 512;
    const bool mid = t >= (L << lgH);
    const int l = mid ? t - (L << lgH) : t >> lgH;
    const int k = mid ? (M >> 1) : t & ((M >> 1) - 1);
    const int64_t line = line0 + l;
    xk[q] = xm[q] = czero<C>();
    if (t < L * P && line < nlines) {
      xk[q] = srcb[line * nzh + k];
      xm[q] = srcb[line * nzh + (M - k)];
    }
  }
#pragma unroll
  for (int q = 0; q < kBatch; ++q) {
    const int t = threadIdx.x + q * 512;
    if (t >= L * P) break;
    const bool mid = t >= (L << lgH);
    const int l = mid ? t - (L << lgH) : t >> lgH;
    const int k = mid ? (M >> 1) : t & ((M >> 1) - 1);
    C Xk = xk[q], Xm = xm[q];
    if (k == 0) {
      Xk.y = 0;
      Xm.y = 0;
    }
    C A, D;
    A.x = Xk.x + Xm.x;
    A.y = Xk.y - Xm.y;
    D.x = Xk.x - Xm.x;
    D.y = Xk.y + Xm.y;
    const C w = __ldg(&tw[k]);
    sm[lay.idx(k, l)] = cadd(A, cmuli(cmul(cconj(w), D)));
    if (k != 0 && k != M - k) sm[lay.idx(M - k, l)] = cadd(cconj(A), cmuli(cmul(w, cconj(D))));
  }
  __syncthreads();
  passes_ct<true, LGM, 0, Plan<LGM>::npass - 1>(sm, lay, tw, 2);
  C* dst = reinterpret_cast<C*>(out.p[comp]) + line0 * M;
  const int nvalid = (int)min((int64_t)L, nlines - line0);
  last_pass_to<true, LGM>(sm, lay, tw, 2, [&](int l, int e, C v) {
    if (l < nvalid) dst[l * M + e] = v;
  });
}

// In-place C2C of length N = 2^LGN along a strided axis: element e of column col of outer line o
// of component c at p[c] + o * os + e * es + col.  A CTA takes W = 2^LGW adjacent columns
// (element-major tile, rows of W elements coalesced); pass 0 takes its inputs from global memory
// and the last pass writes back to it.
// resident CTAs per SM the register cap is set for: ~1280 threads (FP32, 48 registers) or 1024 (FP64, 64)
template <int T, int C_BYTES>
struct StridedMinBlocks {
  static constexpr int raw = (C_BYTES == 16 ? 1024 : 1280) / T;
  static constexpr int value = raw < 1 ? 1 : (raw > 16 ? 16 : raw);
};

template <bool INV, class C, int LGN, int LGW>
__global__ void __launch_bounds__((1 << (LGN + LGW)) / 8, (StridedMinBlocks<(1 << (LGN + LGW)) / 8, sizeof(C)>::value))
    fft_strided_kernel(CP6<C> data, int64_t es, int64_t os, int ncols, const C* __restrict__ tw) {
  constexpr int N = 1 << LGN, W = 1 << LGW, nb = N / 8;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  const LayCol lay{LGW};
  const int comp = blockIdx.z;
  const int col0 = blockIdx.x * W;
  C* base = data.p[comp] + (int64_t)blockIdx.y * os + col0;
  const int wv = min(W, ncols - col0);
  const int w = threadIdx.x & (W - 1), j = threadIdx.x >> LGW;
  C v[8];
  {
    const C* src = base + j * es + w;
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = w < wv ? src[r * nb * es] : czero<C>();
  }
  if constexpr (LGN == 3) {  // one radix-8 pass: registers to global memory
    dft<8, INV>(v);
    if (w < wv) {
#pragma unroll
      for (int r = 0; r < 8; ++r) base[r * es + w] = v[r];
    }
  } else {
    pass0_from_regs<INV>(sm, lay, v, j, w);
    passes_ct<INV, LGN, 1, Plan<LGN>::npass - 1>(sm, lay, tw, 1);
    last_pass_to<INV, LGN>(sm, lay, tw, 1, [&](int l, int e, C val) {
      if (l < wv) base[e * es + l] = val;
    });
  }
}

// log2 of the columns per CTA of the strided passes (measured: 16 and 8 equal, 32 slower)
constexpr int strided_lgw(int lgN) { return lgN >= 10 ? 3 : 4; }

template <class C>
using StridedFn = void (*)(CP6<C>, int64_t, int64_t, int, const C*);

template <bool INV, class C, int LGN>
StridedFn<C> strided_at() {
  return fft_strided_kernel<INV, C, LGN, strided_lgw(LGN)>;
}

// the kernel for N = 2^lgN (8 <= N <= 1024)
template <bool INV, class C>
StridedFn<C> strided_fn(int lgN) {
  switch (lgN) {
    case 3: return strided_at<INV, C, 3>();
    case 4: return strided_at<INV, C, 4>();
    case 5: return strided_at<INV, C, 5>();
    case 6: return strided_at<INV, C, 6>();
    case 7: return strided_at<INV, C, 7>();
    case 8: return strided_at<INV, C, 8>();
    case 9: return strided_at<INV, C, 9>();
    case 10: return strided_at<INV, C, 10>();
  }
  return nullptr;
}

template <class T>
using ZR2CFn = void (*)(CRP6<T>, CP6<typename Cplx<T>::type>, int64_t, const typename Cplx<T>::type*);
template <class T>
using ZC2RFn = void (*)(CP6<typename Cplx<T>::type>, RP6<T>, int64_t, const typename Cplx<T>::type*);

// the z kernels for M = Nz / 2 = 2^lgM (8 <= M <= 512)
template <class T>
ZR2CFn<T> z_r2c_fn(int lgM) {
  switch (lgM) {
    case 3: return fft_z_r2c_kernel<T, 3>;
    case 4: return fft_z_r2c_kernel<T, 4>;
    case 5: return fft_z_r2c_kernel<T, 5>;
    case 6: return fft_z_r2c_kernel<T, 6>;
    case 7: return fft_z_r2c_kernel<T, 7>;
    case 8: return fft_z_r2c_kernel<T, 8>;
    case 9: return fft_z_r2c_kernel<T, 9>;
  }
  return nullptr;
}
template <class T>
ZC2RFn<T> z_c2r_fn(int lgM) {
  switch (lgM) {
    case 3: return fft_z_c2r_kernel<T, 3>;
    case 4: return fft_z_c2r_kernel<T, 4>;
    case 5: return fft_z_c2r_kernel<T, 5>;
    case 6: return fft_z_c2r_kernel<T, 6>;
    case 7: return fft_z_c2r_kernel<T, 7>;
    case 8: return fft_z_c2r_kernel<T, 8>;
    case 9: return fft_z_c2r_kernel<T, 9>;
  }
  return nullptr;
}

template <class C> const C* twiddles(const pic_ctx* ctx, int a);
template <> const double2* twiddles<double2>(const pic_ctx* ctx, int a) { return ctx->twid[a]; }
template <> const float2* twiddles<float2>(const pic_ctx* ctx, int a) { return ctx->twid32[a]; }

template <class C>
pic_status launch_strided(pic_ctx* ctx, CP6<C> d, int axis, bool inv, int ncomp) {
  const int N = (int)ctx->N[axis];
  const int lgN = __builtin_ctz((unsigned)N);
  const int W = 1 << strided_lgw(lgN);
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
  StridedFn<C> fn = inv ? strided_fn<true, C>(lgN) : strided_fn<false, C>(lgN);
  if (!fn) return pic_set_error(ctx, PIC_ERR_UNSUPPORTED, "transform length %d", N);
  dim3 grid((nzh + W - 1) / W, (unsigned)nouter, ncomp);
  const size_t smem = N > 8 ? (size_t)W * N * sizeof(C) : 0;
  fn<<<grid, W * N / 8, smem, ctx->stream>>>(d, es, os, nzh, twiddles<C>(ctx, axis));
  PIC_LAUNCH_CHECK(ctx);
  return PIC_OK;
}

int z_lines_per_cta(int Nz) { return kZTile / (Nz / 2); }

template <class T>
pic_status set_smem_attrs(pic_ctx* ctx) {
  using C = typename Cplx<T>::type;
  for (int lgM = 3; lgM <= 9; ++lgM) {
    const int zsm = (kZTile >> lgM) * zline_len(1 << lgM) * (int)sizeof(C);
    PIC_CUDA_TRY(ctx, cudaFuncSetAttribute(z_r2c_fn<T>(lgM), cudaFuncAttributeMaxDynamicSharedMemorySize, zsm));
    PIC_CUDA_TRY(ctx, cudaFuncSetAttribute(z_c2r_fn<T>(lgM), cudaFuncAttributeMaxDynamicSharedMemorySize, zsm));
  }
  for (int lgN = 4; lgN <= 10; ++lgN) {
    const int ssm = (1 << (lgN + strided_lgw(lgN))) * (int)sizeof(C);
    PIC_CUDA_TRY(ctx, cudaFuncSetAttribute(strided_fn<false, C>(lgN), cudaFuncAttributeMaxDynamicSharedMemorySize, ssm));
    PIC_CUDA_TRY(ctx, cudaFuncSetAttribute(strided_fn<true, C>(lgN), cudaFuncAttributeMaxDynamicSharedMemorySize, ssm));
  }
  return PIC_OK;
}

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
    float2* hf = new float2[N];
    for (int64_t j = 0; j < N; ++j) {
      double s, c;
      sincospi_frac(2 * j, N, &s, &c);
      h[j] = make_double2(c, -s);  // exp(-2 pi i j / N)
      hf[j] = make_float2((float)c, (float)-s);
    }
    cudaError_t e = cudaMalloc(&ctx->twid[a], N * sizeof(double2));
    if (e == cudaSuccess) e = cudaMemcpy(ctx->twid[a], h, N * sizeof(double2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->twid32[a], N * sizeof(float2));
    if (e == cudaSuccess) e = cudaMemcpy(ctx->twid32[a], hf, N * sizeof(float2), cudaMemcpyHostToDevice);
    delete[] h;
    delete[] hf;
    if (e != cudaSuccess) return pic_set_error(ctx, PIC_ERR_NOMEM, "twiddle table: %s", cudaGetErrorString(e));
  }
  pic_status st = set_smem_attrs<double>(ctx);
  if (st != PIC_OK) return st;
  return set_smem_attrs<float>(ctx);
}

template <class T>
pic_status fft_r2c(pic_ctx* ctx, CRP6<T> in, CP6<typename Cplx<T>::type> out, int ncomp) {
  using C = typename Cplx<T>::type;
  const int Nz = (int)ctx->N[2];
  const int L = z_lines_per_cta(Nz);
  const int64_t nlines = ctx->N[0] * ctx->N[1];
  ZR2CFn<T> fn = z_r2c_fn<T>(__builtin_ctz((unsigned)(Nz / 2)));
  if (!fn) return pic_set_error(ctx, PIC_ERR_UNSUPPORTED, "transform length %d", Nz);
  dim3 grid((unsigned)((nlines + L - 1) / L), ncomp);
  const size_t smem = (size_t)L * zline_len(Nz / 2) * sizeof(C);
  fn<<<grid, kZTile / 8, smem, ctx->stream>>>(in, out, nlines, twiddles<C>(ctx, 2));
  PIC_LAUNCH_CHECK(ctx);
  pic_status st = launch_strided<C>(ctx, out, 1, false, ncomp);
  if (st != PIC_OK) return st;
  return launch_strided<C>(ctx, out, 0, false, ncomp);
}

template <class T>
pic_status fft_c2r(pic_ctx* ctx, CP6<typename Cplx<T>::type> in, RP6<T> out, int ncomp) {
  using C = typename Cplx<T>::type;
  pic_status st = launch_strided<C>(ctx, in, 0, true, ncomp);
  if (st != PIC_OK) return st;
  st = launch_strided<C>(ctx, in, 1, true, ncomp);
  if (st != PIC_OK) return st;
  const int Nz = (int)ctx->N[2];
  const int L = z_lines_per_cta(Nz);
  const int64_t nlines = ctx->N[0] * ctx->N[1];
  ZC2RFn<T> fn = z_c2r_fn<T>(__builtin_ctz((unsigned)(Nz / 2)));
  if (!fn) return pic_set_error(ctx, PIC_ERR_UNSUPPORTED, "transform length %d", Nz);
  dim3 grid((unsigned)((nlines + L - 1) / L), ncomp);
  const size_t smem = (size_t)L * zline_len(Nz / 2) * sizeof(C);
  fn<<<grid, kZTile / 8, smem, ctx->stream>>>(in, out, nlines, twiddles<C>(ctx, 2));
  PIC_LAUNCH_CHECK(ctx);
  return PIC_OK;
}

template pic_status fft_r2c<double>(pic_ctx*, CRP6<double>, CP6<double2>, int);
template pic_status fft_r2c<float>(pic_ctx*, CRP6<float>, CP6<float2>, int);
template pic_status fft_c2r<double>(pic_ctx*, CP6<double2>, RP6<double>, int);
template pic_status fft_c2r<float>(pic_ctx*, CP6<float2>, RP6<float>, int);
