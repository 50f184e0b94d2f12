// Vector operations of the GCR solver on internal spinor layouts:
// norms and inner products (two-stage, fixed-order reductions: the same
// inputs always give the same bits), complex axpy with per-RHS
// coefficients read from device memory, scaling and precision conversion.
//
// A spinor of either precision is viewed as 6 V "pairs" of complex numbers:
// pair (k, s) holds components 2k and 2k+1 of site s.  FP32 stores a pair as
// one float4 at k*V + s; FP64 as two double2 at 2k*V + s and (2k+1)*V + s.
#include <type_traits>

#include "qcd_internal.cuh"

namespace {

constexpr int RED_TPB = 256;

struct PD {  // FP64 pair access
  using R = double;
  static constexpr size_t bytes = 192;
  static __device__ inline void ld(const char* b, int V, int k, int s, Cplx<double>& a, Cplx<double>& c) {
    const double2* p = (const double2*)b;
    double2 x = p[(size_t)(2 * k) * V + s], y = p[(size_t)(2 * k + 1) * V + s];
    a = cmk(x.x, x.y);
    c = cmk(y.x, y.y);
  }
  static __device__ inline void st(char* b, int V, int k, int s, Cplx<double> a, Cplx<double> c) {
    double2* p = (double2*)b;
    p[(size_t)(2 * k) * V + s] = make_double2(a.re, a.im);
    p[(size_t)(2 * k + 1) * V + s] = make_double2(c.re, c.im);
  }
};
struct PF {  // FP32 pair access
  using R = float;
  static constexpr size_t bytes = 96;
  static __device__ inline void ld(const char* b, int V, int k, int s, Cplx<float>& a, Cplx<float>& c) {
    float4 v = ((const float4*)b)[(size_t)k * V + s];
    a = cmk(v.x, v.y);
    c = cmk(v.z, v.w);
  }
  static __device__ inline void st(char* b, int V, int k, int s, Cplx<float> a, Cplx<float> c) {
    ((float4*)b)[(size_t)k * V + s] = make_float4(a.re, a.im, c.re, c.im);
  }
};

// Whole-site access (all 12 components), the form the site-major kernels use.
template <typename X>
__device__ inline void ld_site(const char* b, int V, int s, Cplx<typename X::R> (&a)[12]) {
#pragma unroll
  for (int q = 0; q < 6; q++) X::ld(b, V, q, s, a[2 * q], a[2 * q + 1]);
}
template <typename X>
__device__ inline void st_site(char* b, int V, int s, const Cplx<typename X::R> (&a)[12]) {
#pragma unroll
  for (int q = 0; q < 6; q++) X::st(b, V, q, s, a[2 * q], a[2 * q + 1]);
}
struct PH {  // FP16 + per-site scale (FieldsH layout); whole-site access only
  using R = float;
  static constexpr size_t bytes = FieldsH::spinor_bytes;
};
template <>
__device__ inline void ld_site<PH>(const char* b, int V, int s, Cplx<float> (&a)[12]) {
  const Spinor<float> v = FieldsH::load_spinor(b, V, s);
#pragma unroll
  for (int q = 0; q < 12; q++) a[q] = v.c[q];
}
template <>
__device__ inline void st_site<PH>(char* b, int V, int s, const Cplx<float> (&a)[12]) {
  Spinor<float> v;
#pragma unroll
  for (int q = 0; q < 12; q++) v.c[q] = a[q];
  FieldsH::store_spinor(b, V, s, v);
}
// store a, then a <- the values a later load returns (a changes only for PH)
template <typename X>
__device__ inline void st_site_rounded(char* b, int V, int s, Cplx<typename X::R> (&a)[12]) {
  st_site<X>(b, V, s, a);
}
template <>
__device__ inline void st_site_rounded<PH>(char* b, int V, int s, Cplx<float> (&a)[12]) {
  Spinor<float> v;
#pragma unroll
  for (int q = 0; q < 12; q++) v.c[q] = a[q];
  uint2 w[6];
  float sc;
  FieldsH::encode(v, w, sc);
  uint2* p = (uint2*)b;
#pragma unroll
  for (int k = 0; k < 6; k++) p[(size_t)k * V + s] = w[k];
  ((float*)FieldsH::scale_ptr(b, V))[s] = sc;
  v = FieldsH::decode(w, sc);
#pragma unroll
  for (int q = 0; q < 12; q++) a[q] = v.c[q];
}

// arithmetic type of a mixed product: FP32 only when both sides are FP32
template <typename X, typename Y>
struct Acc { using R = double; };
template <>
struct Acc<PF, PF> { using R = float; };
template <>
struct Acc<PH, PF> { using R = float; };
template <>
struct Acc<PH, PH> { using R = float; };

__device__ inline double2 warp_sum(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// block-wide sum in a fixed order; result valid in thread 0
__device__ inline double2 block_sum(double2 v) {
  __shared__ double2 sh[32];
  v = warp_sum(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double2 t = make_double2(0, 0);
  if (w == 0) {
    int nw = (blockDim.x + 31) >> 5;
    t = l < nw ? sh[l] : make_double2(0, 0);
    t = warp_sum(t);
  }
  return t;
}

// OP 0: sum |x|^2 ; OP 1: sum conj(x) y
template <typename X, typename Y, int OP>
__global__ void __launch_bounds__(RED_TPB) k_reduce(const char* __restrict__ x, const char* __restrict__ y, int V,
                                                    double2* __restrict__ part, const int* mask) {
  const int rhs = blockIdx.y;
  double2 acc = make_double2(0, 0);
  if (!mask || mask[rhs]) {
    using R = typename Acc<X, Y>::R;
    const char* xb = x + (size_t)rhs * X::bytes * V;
    const char* yb = OP ? y + (size_t)rhs * Y::bytes * V : nullptr;
    R tr = 0, ti = 0;   // per-thread sums, widened once
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < V; s += gridDim.x * blockDim.x) {
      R sr = 0, si = 0;
#pragma unroll
      for (int k = 0; k < 6; k++) {
        Cplx<typename X::R> a, b;
        X::ld(xb, V, k, s, a, b);
        if (OP == 0) {
          sr += (R)a.re * (R)a.re + (R)a.im * (R)a.im + (R)b.re * (R)b.re + (R)b.im * (R)b.im;
        } else {
          Cplx<typename Y::R> c, d;
          Y::ld(yb, V, k, s, c, d);
          sr += (R)a.re * (R)c.re + (R)a.im * (R)c.im + (R)b.re * (R)d.re + (R)b.im * (R)d.im;
          si += (R)a.re * (R)c.im - (R)a.im * (R)c.re + (R)b.re * (R)d.im - (R)b.im * (R)d.re;
        }
      }
      tr += sr;
      ti += si;
    }
    acc = make_double2((double)tr, (double)ti);
  }
  double2 t = block_sum(acc);
  if (threadIdx.x == 0) part[(size_t)rhs * gridDim.x + blockIdx.x] = t;
}

// sum the G partials of each rhs in a fixed order
__global__ void __launch_bounds__(RED_TPB) k_reduce_final(const double2* __restrict__ part, int G, double2* out,
                                                          int cplx, const int* mask) {
  const int rhs = blockIdx.x;
  if (mask && !mask[rhs]) return;
  double2 acc = make_double2(0, 0);
  for (int i = threadIdx.x; i < G; i += blockDim.x) {
    double2 v = part[(size_t)rhs * G + i];
    acc.x += v.x;
    acc.y += v.y;
  }
  double2 t = block_sum(acc);
  if (threadIdx.x == 0) {
    if (cplx)
      out[rhs] = t;
    else
      ((double*)out)[rhs] = t.x;
  }
}

int red_grid(const qcd_ctx* c) {
  int g = (c->g.V + RED_TPB - 1) / RED_TPB;
  return g < 4 * 152 ? g : 4 * 152;
}

template <typename X, typename Y, int OP>
qcd_status reduce(qcd_ctx* c, const void* x, const void* y, int nrhs, void* out, const int* mask) {
  int G = red_grid(c);
  QCD_TRY(devbuf_ensure(c->red, (size_t)G * nrhs * sizeof(double2)));
  ProfScope ps(c, FAM_BLAS, (double)c->g.V * nrhs * (X::bytes + (OP ? Y::bytes : 0)), (double)c->g.V * nrhs * 96, 2);
  k_reduce<X, Y, OP><<<dim3(G, nrhs), RED_TPB, 0, c->stream>>>((const char*)x, (const char*)y, c->g.V,
                                                                (double2*)c->red.p, mask);
  k_reduce_final<<<nrhs, RED_TPB, 0, c->stream>>>((const double2*)c->red.p, G, (double2*)out, OP, mask);
  QCD_CUDA_OK(cudaGetLastError());
  return QCD_OK;
}

// y_r += sign * sum_j coef[j*nrhs + r] * x_{j,r}
template <typename Y, typename X>
__global__ void k_multi_caxpy(char* __restrict__ y, const char* __restrict__ xbase, int nx, size_t xstride,
                              const double2* __restrict__ coef, double sign, int V, int nrhs, const int* mask) {
  const int rhs = blockIdx.y;
  if (mask && !mask[rhs]) return;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  using R = typename Y::R;
  char* yb = y + (size_t)rhs * Y::bytes * V;
#pragma unroll 1
  for (int k = 0; k < 6; k++) {
    Cplx<R> a, b;
    Y::ld(yb, V, k, s, a, b);
    Cplx<double> ad = cmk((double)a.re, (double)a.im), bd = cmk((double)b.re, (double)b.im);
    for (int j = 0; j < nx; j++) {
      double2 cf = coef[(size_t)j * nrhs + rhs];
      Cplx<double> w = cmk(sign * cf.x, sign * cf.y);
      Cplx<typename X::R> u, v;
      X::ld(xbase + j * xstride + (size_t)rhs * X::bytes * V, V, k, s, u, v);
      ad = ad + w * cmk((double)u.re, (double)u.im);
      bd = bd + w * cmk((double)v.re, (double)v.im);
    }
    Y::st(yb, V, k, s, cmk((R)ad.re, (R)ad.im), cmk((R)bd.re, (R)bd.im));
  }
}

// FP32 specialisation: coefficients applied in FP32
template <>
__global__ void k_multi_caxpy<PF, PF>(char* __restrict__ y, const char* __restrict__ xbase, int nx, size_t xstride,
                                      const double2* __restrict__ coef, double sign, int V, int nrhs,
                                      const int* mask) {
  const int rhs = blockIdx.y;
  if (mask && !mask[rhs]) return;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  float4* yb = (float4*)(y + (size_t)rhs * PF::bytes * V);
#pragma unroll 1
  for (int k = 0; k < 6; k++) {
    float4 a = yb[(size_t)k * V + s];
    for (int j = 0; j < nx; j++) {
      double2 cf = coef[(size_t)j * nrhs + rhs];
      float wr = (float)(sign * cf.x), wi = (float)(sign * cf.y);
      float4 u = ((const float4*)(xbase + j * xstride + (size_t)rhs * PF::bytes * V))[(size_t)k * V + s];
      a.x += wr * u.x - wi * u.y;
      a.y += wr * u.y + wi * u.x;
      a.z += wr * u.z - wi * u.w;
      a.w += wr * u.w + wi * u.z;
    }
    yb[(size_t)k * V + s] = a;
  }
}

template <typename X>
__global__ void k_scale(char* __restrict__ x, const double* __restrict__ sc, int V, int nrhs, const int* mask) {
  const int rhs = blockIdx.y;
  if (mask && !mask[rhs]) return;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  using R = typename X::R;
  R f = (R)sc[rhs];
  char* xb = x + (size_t)rhs * X::bytes * V;
#pragma unroll
  for (int k = 0; k < 6; k++) {
    Cplx<R> a, b;
    X::ld(xb, V, k, s, a, b);
    X::st(xb, V, k, s, f * a, f * b);
  }
}

// out = x - y (same precision)
template <typename X>
__global__ void k_xmy(const char* __restrict__ x, const char* __restrict__ y, char* __restrict__ out, int V, int nrhs,
                      const int* mask) {
  const int rhs = blockIdx.y;
  if (mask && !mask[rhs]) return;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  size_t off = (size_t)rhs * X::bytes * V;
#pragma unroll
  for (int k = 0; k < 6; k++) {
    Cplx<typename X::R> a, b, c, d;
    X::ld(x + off, V, k, s, a, b);
    X::ld(y + off, V, k, s, c, d);
    X::st(out + off, V, k, s, a - c, b - d);
  }
}

template <typename I, typename O>
__global__ void k_convert(const char* __restrict__ in, char* __restrict__ out, int V, int nrhs, const int* mask) {
  const int rhs = blockIdx.y;
  if (mask && !mask[rhs]) return;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  using RO = typename O::R;
#pragma unroll
  for (int k = 0; k < 6; k++) {
    Cplx<typename I::R> a, b;
    I::ld(in + (size_t)rhs * I::bytes * V, V, k, s, a, b);
    O::st(out + (size_t)rhs * O::bytes * V, V, k, s, cmk((RO)a.re, (RO)a.im), cmk((RO)b.re, (RO)b.im));
  }
}

inline dim3 grid2(const qcd_ctx* c, int nrhs) { return dim3((c->g.V + 255) / 256, nrhs); }
// ---------------------------------------------------------------------------
// Fused Gram-Schmidt step of the GCR solver
// ---------------------------------------------------------------------------
constexpr int GS_TPB = 256;

// block sum of NV doubles; thread 0 holds the result in out[]
template <int NV>
__device__ inline void block_sum_n(double (&v)[NV], double* sh /* [NV][32] */) {
#pragma unroll
  for (int k = 0; k < NV; k++)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (l == 0)
#pragma unroll
    for (int k = 0; k < NV; k++) sh[k * 32 + w] = v[k];
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NV; k++) {
      double t = 0;
      for (int ww = 0; ww < nw; ww++) t += sh[k * 32 + ww];
      v[k] = t;
    }
}

// dots[j][r] = (chi_j, chi_k) for j < k: chi_k is read once, each chi_j once.
// One thread per site; per-j CTA sums go to part[r][j][cta].
template <typename X>
__global__ void __launch_bounds__(GS_TPB) k_multi_dot(const char* __restrict__ chi, size_t jstride, int k, int V,
                                                       double2* __restrict__ part, const int* mask) {
  __shared__ double sh[2 * 32];
  const int rhs = blockIdx.y;
  if (mask && !mask[rhs]) return;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const size_t roff = (size_t)rhs * X::bytes * V;
  using R = typename X::R;
  Cplx<R> ck[12];
  if (s < V) {
#pragma unroll
    for (int q = 0; q < 6; q++) X::ld(chi + k * jstride + roff, V, q, s, ck[2 * q], ck[2 * q + 1]);
  } else {
#pragma unroll
    for (int q = 0; q < 12; q++) ck[q] = cmk((R)0, (R)0);
  }
  for (int j = 0; j < k; j++) {
    R sr = 0, si = 0;
    if (s < V) {
#pragma unroll
      for (int q = 0; q < 6; q++) {
        Cplx<R> a, b;
        X::ld(chi + j * jstride + roff, V, q, s, a, b);
        sr += a.re * ck[2 * q].re + a.im * ck[2 * q].im + b.re * ck[2 * q + 1].re + b.im * ck[2 * q + 1].im;
        si += a.re * ck[2 * q].im - a.im * ck[2 * q].re + b.re * ck[2 * q + 1].im - b.im * ck[2 * q + 1].re;
      }
    }
    double v[2] = {(double)sr, (double)si};
    block_sum_n<2>(v, sh);
    if (threadIdx.x == 0) part[((size_t)rhs * k + j) * gridDim.x + blockIdx.x] = make_double2(v[0], v[1]);
  }
}

// Same result with per-thread register accumulators: each thread walks its
// sites (grid-stride) keeping one accumulator per j, so the CTA reduction
// happens once per j per CTA instead of once per j per 256 sites.
template <typename X, int KMAX>
__global__ void __launch_bounds__(GS_TPB) k_multi_dot_acc(const char* __restrict__ chi, size_t jstride, int k, int V,
                                                           double2* __restrict__ part, const int* mask) {
  __shared__ double sh[2 * 32];
  const int rhs = blockIdx.y;
  if (mask && !mask[rhs]) return;
  using R = typename X::R;
  const size_t roff = (size_t)rhs * X::bytes * V;
  R ar[KMAX], ai[KMAX];
#pragma unroll
  for (int j = 0; j < KMAX; j++) ar[j] = ai[j] = (R)0;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < V; s += gridDim.x * blockDim.x) {
    Cplx<R> ck[12];
    ld_site<X>(chi + k * jstride + roff, V, s, ck);
#pragma unroll
    for (int j = 0; j < KMAX; j++) {
      if (j < k) {
        Cplx<R> u[12];
        ld_site<X>(chi + j * jstride + roff, V, s, u);
        Cplx<R> d = cmk((R)0, (R)0);
#pragma unroll
        for (int q = 0; q < 12; q++) cmac_conj(d, u[q], ck[q]);
        ar[j] += d.re;
        ai[j] += d.im;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < KMAX; j++) {
    if (j < k) {
      double v[2] = {(double)ar[j], (double)ai[j]};
      block_sum_n<2>(v, sh);
      if (threadIdx.x == 0) part[((size_t)rhs * k + j) * gridDim.x + blockIdx.x] = make_double2(v[0], v[1]);
    }
  }
}

// out[j*nrhs + r] = sum over g of part[r][j][g] (fixed order)
__global__ void __launch_bounds__(RED_TPB) k_sum_parts(const double2* __restrict__ part, int nj, int G,
                                                       double2* __restrict__ out, int nrhs, const int* mask) {
  const int j = blockIdx.x, rhs = blockIdx.y;
  if (mask && !mask[rhs]) return;
  double2 acc = make_double2(0, 0);
  for (int i = threadIdx.x; i < G; i += blockDim.x) {
    double2 v = part[((size_t)rhs * nj + j) * G + i];
    acc.x += v.x;
    acc.y += v.y;
  }
  double2 t = block_sum(acc);
  if (threadIdx.x == 0) out[(size_t)j * nrhs + rhs] = t;
}

// chi_k -= sum_{j<k} dots[j] chi_j; then partial sums of |chi_k|^2 and (chi_k, rho)
template <typename X>
__global__ void __launch_bounds__(GS_TPB) k_gs_orth(char* __restrict__ chi, size_t jstride, int k,
                                                     const double2* __restrict__ dots, const char* __restrict__ rho,
                                                     int V, int nrhs, double2* __restrict__ part, const int* mask) {
  __shared__ double sh[3 * 32];
  const int rhs = blockIdx.y;
  if (mask && !mask[rhs]) return;
  using R = typename X::R;
  const size_t roff = (size_t)rhs * X::bytes * V;
  char* ckp = chi + k * jstride + roff;
  const char* rp = rho + (size_t)rhs * PD::bytes * V;
  double n2 = 0, cr = 0, ci = 0;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < V; s += gridDim.x * blockDim.x) {
#pragma unroll 1
    for (int q = 0; q < 6; q++) {
      Cplx<R> a, b;
      X::ld(ckp, V, q, s, a, b);
      for (int j = 0; j < k; j++) {
        double2 d = dots[(size_t)j * nrhs + rhs];
        Cplx<R> w = cmk((R)d.x, (R)d.y), u, v;
        X::ld(chi + j * jstride + roff, V, q, s, u, v);
        a = a - w * u;
        b = b - w * v;
      }
      X::st(ckp, V, q, s, a, b);
      Cplx<double> x, y;
      PD::ld(rp, V, q, s, x, y);
      n2 += (double)(a.re * a.re + a.im * a.im + b.re * b.re + b.im * b.im);
      cr += (double)a.re * x.re + (double)a.im * x.im + (double)b.re * y.re + (double)b.im * y.im;
      ci += (double)a.re * x.im - (double)a.im * x.re + (double)b.re * y.im - (double)b.im * y.re;
    }
  }
  double v[3] = {n2, cr, ci};
  block_sum_n<3>(v, sh);
  if (threadIdx.x == 0) {
    double2* p = part + (size_t)rhs * 2 * gridDim.x;
    p[blockIdx.x] = make_double2(v[0], 0.0);
    p[gridDim.x + blockIdx.x] = make_double2(v[1], v[2]);
  }
}

// Site-major form of k_gs_orth: a thread holds all 12 components of chi_k
// for its site and walks the j < k vectors with independent loads (the j
// loop is unrolled to KMAX), so many loads are in flight per thread.
template <typename X, typename RH, int KMAX>
__global__ void __launch_bounds__(GS_TPB) k_gs_orth_sm(char* __restrict__ chi, size_t jstride, int k,
                                                        const double2* __restrict__ dots, const char* __restrict__ rho,
                                                        int V, int nrhs, double2* __restrict__ part, const int* mask) {
  __shared__ double sh[3 * 32];
  __shared__ float2 w_s[KMAX];
  const int rhs = blockIdx.y;
  if (mask && !mask[rhs]) return;
  using R = typename X::R;
  if (threadIdx.x < KMAX && (int)threadIdx.x < k) {
    double2 d = dots[(size_t)threadIdx.x * nrhs + rhs];
    w_s[threadIdx.x] = make_float2((float)d.x, (float)d.y);
  }
  __syncthreads();
  const size_t roff = (size_t)rhs * X::bytes * V;
  char* ckp = chi + k * jstride + roff;
  const char* rp = rho + (size_t)rhs * RH::bytes * V;
  // per-thread sums in the arithmetic type of the pair (FP32 unless FP64 is
  // involved), widened to FP64 once per thread: FP64 arithmetic per site
  // would make the pass ALU-bound on this GPU
  using A = typename Acc<X, RH>::R;
  A n2 = 0, cr = 0, ci = 0;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < V; s += gridDim.x * blockDim.x) {
    Cplx<R> a[12];
    ld_site<X>(ckp, V, s, a);
#pragma unroll
    for (int j = 0; j < KMAX; j++) {
      if (j < k) {
        Cplx<R> u[12];
        ld_site<X>(chi + j * jstride + roff, V, s, u);
        const Cplx<R> mw = cmk((R)-w_s[j].x, (R)-w_s[j].y);
#pragma unroll
        for (int q = 0; q < 12; q++) cmac(a[q], mw, u[q]);
      }
    }
    st_site_rounded<X>(ckp, V, s, a);   // norm and overlap with rho of chi_k as stored
    Cplx<typename RH::R> x[12];
    ld_site<RH>(rp, V, s, x);
#pragma unroll
    for (int q = 0; q < 12; q++) {
      const A ar = (A)a[q].re, ai = (A)a[q].im, xr = (A)x[q].re, xi = (A)x[q].im;
      n2 = rfma(ar, ar, n2);
      n2 = rfma(ai, ai, n2);
      cr = rfma(ar, xr, cr);
      cr = rfma(ai, xi, cr);
      ci = rfma(ar, xi, ci);
      ci = rfma(-ai, xr, ci);
    }
  }
  double v[3] = {(double)n2, (double)cr, (double)ci};
  block_sum_n<3>(v, sh);
  if (threadIdx.x == 0) {
    double2* pp = part + (size_t)rhs * 2 * gridDim.x;
    pp[blockIdx.x] = make_double2(v[0], 0.0);
    pp[gridDim.x + blockIdx.x] = make_double2(v[1], v[2]);
  }
}

// Site-major y (FP64) += sign sum_{j<nx} coef_j x_j (FP32)
template <int KMAX>
__global__ void __launch_bounds__(GS_TPB) k_caxpy_sm(char* __restrict__ y, const char* __restrict__ xbase, int nx,
                                                      size_t xstride, const double2* __restrict__ coef, double sign,
                                                      int V, int nrhs, const int* mask) {
  __shared__ double2 c_s[KMAX];
  const int rhs = blockIdx.y;
  if (mask && !mask[rhs]) return;
  if (threadIdx.x < KMAX && (int)threadIdx.x < nx) {
    double2 c = coef[(size_t)threadIdx.x * nrhs + rhs];
    c_s[threadIdx.x] = make_double2(sign * c.x, sign * c.y);
  }
  __syncthreads();
  char* yb = y + (size_t)rhs * PD::bytes * V;
  const size_t xoff = (size_t)rhs * PF::bytes * V;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < V; s += gridDim.x * blockDim.x) {
    // the combination sum_j coef_j x_j in FP32 (the x_j are FP32), then one
    // FP64 add per component: FP64 multiply-adds per basis vector would make
    // the pass ALU-bound on this GPU
    Cplx<float> d[12];
#pragma unroll
    for (int q = 0; q < 12; q++) d[q] = cmk(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < KMAX; j++) {
      if (j < nx) {
        Cplx<float> u[12];
#pragma unroll
        for (int q = 0; q < 6; q++) PF::ld(xbase + j * xstride + xoff, V, q, s, u[2 * q], u[2 * q + 1]);
        const Cplx<float> w = cmk((float)c_s[j].x, (float)c_s[j].y);
#pragma unroll
        for (int q = 0; q < 12; q++) cmac(d[q], w, u[q]);
      }
    }
    Cplx<double> a[12];
#pragma unroll
    for (int q = 0; q < 6; q++) PD::ld(yb, V, q, s, a[2 * q], a[2 * q + 1]);
#pragma unroll
    for (int q = 0; q < 12; q++) a[q] = a[q] + cmk((double)d[q].re, (double)d[q].im);
#pragma unroll
    for (int q = 0; q < 6; q++) PD::st(yb, V, q, s, a[2 * q], a[2 * q + 1]);
  }
}

// chi_k *= inv; rho -= ck * chi_k; chi_k stored as XC, rho in the inner
// precision XR (the same real type); partial |rho|^2
template <typename XC, typename XR>
__global__ void __launch_bounds__(GS_TPB) k_gs_finish_inner(char* __restrict__ chik, const double* __restrict__ inv,
                                                             const double2* __restrict__ ck, char* __restrict__ rho,
                                                             int V, double2* __restrict__ part, const int* mask) {
  __shared__ double sh[32];
  const int rhs = blockIdx.y;
  if (mask && !mask[rhs]) return;
  using R = typename XR::R;
  char* cp = chik + (size_t)rhs * XC::bytes * V;
  char* rp = rho + (size_t)rhs * XR::bytes * V;
  const R f = (R)inv[rhs];
  const Cplx<R> mc = cmk((R)-ck[rhs].x, (R)-ck[rhs].y);
  R n2 = 0;   // per-thread sum, widened once (see k_gs_orth_sm)
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < V; s += gridDim.x * blockDim.x) {
    Cplx<R> a[12], x[12];
    ld_site<XR>(rp, V, s, x);
    if constexpr (std::is_same<XC, PH>::value) {
      // FP16 words unchanged; only the site's scale factor takes the normalisation
      uint2 w[6];
      float sc;
      FieldsH::load_words(cp, V, s, w, sc);
      sc *= (float)f;
      const Spinor<float> v = FieldsH::decode(w, sc);
#pragma unroll
      for (int q = 0; q < 12; q++) a[q] = cmk((R)v.c[q].re, (R)v.c[q].im);
      ((float*)FieldsH::scale_ptr(cp, V))[s] = sc;
    } else {
      ld_site<XC>(cp, V, s, a);
#pragma unroll
      for (int q = 0; q < 12; q++) a[q] = f * a[q];
      st_site<XC>(cp, V, s, a);
    }
    R acc = 0;
#pragma unroll
    for (int q = 0; q < 12; q++) {
      cmac(x[q], mc, a[q]);
      acc += x[q].re * x[q].re + x[q].im * x[q].im;
    }
    st_site<XR>(rp, V, s, x);
    n2 += acc;
  }
  double v[1] = {(double)n2};
  block_sum_n<1>(v, sh);
  if (threadIdx.x == 0) part[(size_t)rhs * gridDim.x + blockIdx.x] = make_double2(v[0], 0.0);
}

}  // namespace

qcd_status blas_norm2(qcd_ctx* c, const void* x, int prec, int nrhs, double* out_dev, const int* mask) {
  if (prec == QCD_PREC_F64) return reduce<PD, PD, 0>(c, x, nullptr, nrhs, out_dev, mask);
  return reduce<PF, PF, 0>(c, x, nullptr, nrhs, out_dev, mask);
}

qcd_status blas_dot(qcd_ctx* c, const void* x, int px, const void* y, int py, int nrhs, double* out_dev,
                    const int* mask) {
  if (px == QCD_PREC_F64 && py == QCD_PREC_F64) return reduce<PD, PD, 1>(c, x, y, nrhs, out_dev, mask);
  if (px == QCD_PREC_F32 && py == QCD_PREC_F64) return reduce<PF, PD, 1>(c, x, y, nrhs, out_dev, mask);
  if (px == QCD_PREC_F64 && py == QCD_PREC_F32) return reduce<PD, PF, 1>(c, x, y, nrhs, out_dev, mask);
  return reduce<PF, PF, 1>(c, x, y, nrhs, out_dev, mask);
}

qcd_status blas_multi_caxpy(qcd_ctx* c, void* y, int py, const void* xbase, int px, int nx, size_t xstride,
                            const double* coef_dev, double sign, int nrhs, const int* mask) {
  if (nx <= 0) return QCD_OK;
  dim3 g = grid2(c, nrhs);
  const double by = py == QCD_PREC_F64 ? 192 : 96, bx = px == QCD_PREC_F64 ? 192 : 96;
  ProfScope ps(c, FAM_BLAS, (double)c->g.V * nrhs * (2 * by + nx * bx), (double)c->g.V * nrhs * nx * 96);
  if (py == QCD_PREC_F64 && px == QCD_PREC_F64)
    k_multi_caxpy<PD, PD><<<g, 256, 0, c->stream>>>((char*)y, (const char*)xbase, nx, xstride,
                                                    (const double2*)coef_dev, sign, c->g.V, nrhs, mask);
  else if (py == QCD_PREC_F64 && px == QCD_PREC_F32) {
    const dim3 gs(red_grid(c), nrhs);
    const double2* cf = (const double2*)coef_dev;
    if (nx <= 8)
      k_caxpy_sm<8><<<gs, GS_TPB, 0, c->stream>>>((char*)y, (const char*)xbase, nx, xstride, cf, sign, c->g.V, nrhs,
                                                  mask);
    else if (nx <= 16)
      k_caxpy_sm<16><<<gs, GS_TPB, 0, c->stream>>>((char*)y, (const char*)xbase, nx, xstride, cf, sign, c->g.V,
                                                   nrhs, mask);
    else
      k_caxpy_sm<32><<<gs, GS_TPB, 0, c->stream>>>((char*)y, (const char*)xbase, nx, xstride, cf, sign, c->g.V,
                                                   nrhs, mask);
  }
  else if (py == QCD_PREC_F32 && px == QCD_PREC_F32)
    k_multi_caxpy<PF, PF><<<g, 256, 0, c->stream>>>((char*)y, (const char*)xbase, nx, xstride,
                                                    (const double2*)coef_dev, sign, c->g.V, nrhs, mask);
  else {
    qcd_set_error("multi_caxpy: unsupported precision pair");
    return QCD_ERR_ARG;
  }
  QCD_CUDA_OK(cudaGetLastError());
  return QCD_OK;
}

qcd_status blas_scale(qcd_ctx* c, void* x, int px, const double* sc_dev, int nrhs, const int* mask) {
  dim3 g = grid2(c, nrhs);
  ProfScope ps(c, FAM_BLAS, (double)c->g.V * nrhs * 2 * (px == QCD_PREC_F64 ? 192 : 96), (double)c->g.V * nrhs * 24);
  if (px == QCD_PREC_F64)
    k_scale<PD><<<g, 256, 0, c->stream>>>((char*)x, sc_dev, c->g.V, nrhs, mask);
  else
    k_scale<PF><<<g, 256, 0, c->stream>>>((char*)x, sc_dev, c->g.V, nrhs, mask);
  QCD_CUDA_OK(cudaGetLastError());
  return QCD_OK;
}

qcd_status blas_xmy(qcd_ctx* c, const void* x, const void* y, void* out, int prec, int nrhs, const int* mask) {
  dim3 g = grid2(c, nrhs);
  ProfScope ps(c, FAM_BLAS, (double)c->g.V * nrhs * 3 * (prec == QCD_PREC_F64 ? 192 : 96), (double)c->g.V * nrhs * 24);
  if (prec == QCD_PREC_F64)
    k_xmy<PD><<<g, 256, 0, c->stream>>>((const char*)x, (const char*)y, (char*)out, c->g.V, nrhs, mask);
  else
    k_xmy<PF><<<g, 256, 0, c->stream>>>((const char*)x, (const char*)y, (char*)out, c->g.V, nrhs, mask);
  QCD_CUDA_OK(cudaGetLastError());
  return QCD_OK;
}

qcd_status blas_convert(qcd_ctx* c, const void* in, int pin, void* out, int pout, int nrhs, const int* mask) {
  dim3 g = grid2(c, nrhs);
  ProfScope ps(c, FAM_BLAS, (double)c->g.V * nrhs * ((pin == QCD_PREC_F64 ? 192 : 96) + (pout == QCD_PREC_F64 ? 192 : 96)), 0.0);
  if (pin == QCD_PREC_F64 && pout == QCD_PREC_F32)
    k_convert<PD, PF><<<g, 256, 0, c->stream>>>((const char*)in, (char*)out, c->g.V, nrhs, mask);
  else if (pin == QCD_PREC_F32 && pout == QCD_PREC_F64)
    k_convert<PF, PD><<<g, 256, 0, c->stream>>>((const char*)in, (char*)out, c->g.V, nrhs, mask);
  else if (pin == QCD_PREC_F64 && pout == QCD_PREC_F64)
    k_convert<PD, PD><<<g, 256, 0, c->stream>>>((const char*)in, (char*)out, c->g.V, nrhs, mask);
  else
    k_convert<PF, PF><<<g, 256, 0, c->stream>>>((const char*)in, (char*)out, c->g.V, nrhs, mask);
  QCD_CUDA_OK(cudaGetLastError());
  return QCD_OK;
}

// dots_dev[j][r] = (chi_j, chi_k), j < k
qcd_status blas_gs_dots(qcd_ctx* c, const void* chi, int prec, size_t jstride, int k, int nrhs, double* dots_dev,
                        const int* mask, int nactive) {
  if (k <= 0) return QCD_OK;
  const int G = red_grid(c);
  QCD_TRY(devbuf_ensure(c->red, (size_t)G * k * nrhs * sizeof(double2)));
  const double vb = prec == QCD_PREC_F64 ? 192 : prec == QCD_PREC_H16 ? (double)PH::bytes : 96;
  ProfScope ps(c, FAM_BLAS, (double)c->g.V * nactive * (k + 1) * vb, (double)c->g.V * nactive * k * 48, 2);
  const dim3 grid(G, nrhs);
  const char* cp = (const char*)chi;
  double2* pp = (double2*)c->red.p;
  if (prec == QCD_PREC_H16) {
    if (k <= 8) k_multi_dot_acc<PH, 8><<<grid, GS_TPB, 0, c->stream>>>(cp, jstride, k, c->g.V, pp, mask);
    else if (k <= 16) k_multi_dot_acc<PH, 16><<<grid, GS_TPB, 0, c->stream>>>(cp, jstride, k, c->g.V, pp, mask);
    else k_multi_dot_acc<PH, 32><<<grid, GS_TPB, 0, c->stream>>>(cp, jstride, k, c->g.V, pp, mask);
  } else if (prec == QCD_PREC_F64) {
    if (k <= 8) k_multi_dot_acc<PD, 8><<<grid, GS_TPB, 0, c->stream>>>(cp, jstride, k, c->g.V, pp, mask);
    else if (k <= 16) k_multi_dot_acc<PD, 16><<<grid, GS_TPB, 0, c->stream>>>(cp, jstride, k, c->g.V, pp, mask);
    else k_multi_dot_acc<PD, 32><<<grid, GS_TPB, 0, c->stream>>>(cp, jstride, k, c->g.V, pp, mask);
  } else {
    if (k <= 8) k_multi_dot_acc<PF, 8><<<grid, GS_TPB, 0, c->stream>>>(cp, jstride, k, c->g.V, pp, mask);
    else if (k <= 16) k_multi_dot_acc<PF, 16><<<grid, GS_TPB, 0, c->stream>>>(cp, jstride, k, c->g.V, pp, mask);
    else k_multi_dot_acc<PF, 32><<<grid, GS_TPB, 0, c->stream>>>(cp, jstride, k, c->g.V, pp, mask);
  }
  k_sum_parts<<<dim3(k, nrhs), RED_TPB, 0, c->stream>>>((const double2*)c->red.p, k, G, (double2*)dots_dev, nrhs,
                                                        mask);
  QCD_CUDA_OK(cudaGetLastError());
  return QCD_OK;
}

// chi_k -= sum_j dots[j] chi_j; n2c[0][r] = |chi_k|^2 (re), n2c[1][r] = (chi_k, rho)
qcd_status blas_gs_orth(qcd_ctx* c, void* chi, int prec, size_t jstride, int k, const double* dots_dev,
                        const void* rho, int prho, int nrhs, double* n2c_dev, const int* mask, int nactive) {
  const int G = red_grid(c);
  QCD_TRY(devbuf_ensure(c->red, (size_t)G * 2 * nrhs * sizeof(double2)));
  const double vb = prec == QCD_PREC_F64 ? 192 : prec == QCD_PREC_H16 ? (double)PH::bytes : 96;
  ProfScope ps(c, FAM_BLAS, (double)c->g.V * nactive * ((k + 2) * vb + (prho == QCD_PREC_F64 ? 192 : 96)),
               (double)c->g.V * nactive * (k + 2) * 48, 2);
  const dim3 grid(G, nrhs);
  char* cp = (char*)chi;
  const double2* dp = (const double2*)dots_dev;
  const char* rp = (const char*)rho;
  double2* pp = (double2*)c->red.p;
  if (prec == QCD_PREC_H16) {
    if (prho != QCD_PREC_F32) {
      qcd_set_error("gs_orth: an FP16 basis needs an FP32 residual");
      return QCD_ERR_ARG;
    }
    if (k <= 8) k_gs_orth_sm<PH, PF, 8><<<grid, GS_TPB, 0, c->stream>>>(cp, jstride, k, dp, rp, c->g.V, nrhs, pp, mask);
    else if (k <= 16) k_gs_orth_sm<PH, PF, 16><<<grid, GS_TPB, 0, c->stream>>>(cp, jstride, k, dp, rp, c->g.V, nrhs, pp, mask);
    else k_gs_orth_sm<PH, PF, 32><<<grid, GS_TPB, 0, c->stream>>>(cp, jstride, k, dp, rp, c->g.V, nrhs, pp, mask);
  } else if (prec == QCD_PREC_F64)
    k_gs_orth<PD><<<grid, GS_TPB, 0, c->stream>>>(cp, jstride, k, dp, rp, c->g.V, nrhs, pp, mask);
  else if (prho == QCD_PREC_F64) {
    if (k <= 8) k_gs_orth_sm<PF, PD, 8><<<grid, GS_TPB, 0, c->stream>>>(cp, jstride, k, dp, rp, c->g.V, nrhs, pp, mask);
    else if (k <= 16) k_gs_orth_sm<PF, PD, 16><<<grid, GS_TPB, 0, c->stream>>>(cp, jstride, k, dp, rp, c->g.V, nrhs, pp, mask);
    else k_gs_orth_sm<PF, PD, 32><<<grid, GS_TPB, 0, c->stream>>>(cp, jstride, k, dp, rp, c->g.V, nrhs, pp, mask);
  } else {
    if (k <= 8) k_gs_orth_sm<PF, PF, 8><<<grid, GS_TPB, 0, c->stream>>>(cp, jstride, k, dp, rp, c->g.V, nrhs, pp, mask);
    else if (k <= 16) k_gs_orth_sm<PF, PF, 16><<<grid, GS_TPB, 0, c->stream>>>(cp, jstride, k, dp, rp, c->g.V, nrhs, pp, mask);
    else k_gs_orth_sm<PF, PF, 32><<<grid, GS_TPB, 0, c->stream>>>(cp, jstride, k, dp, rp, c->g.V, nrhs, pp, mask);
  }
  k_sum_parts<<<dim3(2, nrhs), RED_TPB, 0, c->stream>>>((const double2*)c->red.p, 2, G, (double2*)n2c_dev, nrhs,
                                                        mask);
  QCD_CUDA_OK(cudaGetLastError());
  return QCD_OK;
}

// chi_k *= inv; rho -= ck chi_k with rho in the inner precision; rn2[r] = |rho|^2 (double2 .x)
qcd_status blas_gs_finish_inner(qcd_ctx* c, void* chik, int pchi, const double* inv_dev, const double* ck_dev,
                                void* rho, int prho, int nrhs, double* rn2_dev, const int* mask, int nactive) {
  const bool h16 = pchi == QCD_PREC_H16 && prho == QCD_PREC_F32;
  const bool f64 = pchi == QCD_PREC_F64 && prho == QCD_PREC_F64;
  const bool f32 = pchi == QCD_PREC_F32 && prho == QCD_PREC_F32;
  if (!h16 && !f64 && !f32) {
    qcd_set_error("gs_finish: unsupported precision pair");
    return QCD_ERR_ARG;
  }
  const int G = red_grid(c);
  QCD_TRY(devbuf_ensure(c->red, (size_t)G * nrhs * sizeof(double2)));
  const dim3 grid(G, nrhs);
  char* cp = (char*)chik;
  const double2* kp = (const double2*)ck_dev;
  char* rp = (char*)rho;
  double2* pp = (double2*)c->red.p;
  // FP16 basis: chi_k read (words + scale) and only its scale written; rho read and written
  const double bytes = h16 ? PH::bytes + 4.0 + 2 * 96 : 4.0 * (f64 ? 192 : 96);
  ProfScope ps(c, FAM_BLAS, (double)c->g.V * nactive * bytes, (double)c->g.V * nactive * 96, 2);
  if (h16)
    k_gs_finish_inner<PH, PF><<<grid, GS_TPB, 0, c->stream>>>(cp, inv_dev, kp, rp, c->g.V, pp, mask);
  else if (f64)
    k_gs_finish_inner<PD, PD><<<grid, GS_TPB, 0, c->stream>>>(cp, inv_dev, kp, rp, c->g.V, pp, mask);
  else
    k_gs_finish_inner<PF, PF><<<grid, GS_TPB, 0, c->stream>>>(cp, inv_dev, kp, rp, c->g.V, pp, mask);
  k_sum_parts<<<dim3(1, nrhs), RED_TPB, 0, c->stream>>>((const double2*)c->red.p, 1, G, (double2*)rn2_dev, nrhs,
                                                        mask);
  QCD_CUDA_OK(cudaGetLastError());
  return QCD_OK;
}
