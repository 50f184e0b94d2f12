// Internal types, field layouts and device helpers of the Wilson-clover
// library.  Nothing here is part of the public C-ABI (include/qcd.h).
//
// Site order everywhere is lexicographic, s = ((t*LZ + z)*LY + y)*LX + x.
// Internal layouts are structure-of-arrays over sites so that consecutive
// threads (consecutive sites) read consecutive 16-byte words:
//
//   spinor FP64   double2 [rhs][12][V]   component c = 3*spin + colour
//   spinor FP32   float4  [rhs][6][V]    float4 k = components 2k, 2k+1
//   gauge  FP64   double2 [4][9][V]      U_mu(x)[row][col], full matrix
//   gauge  FP32   float4  [4][3][V]      rows 0 and 1; row 2 = conj(r0 x r1)
//   clover FP64   double2 [36][V]        two packed 6x6 Hermitian chiral blocks
//   clover FP32   float4  [18][V]        same 72 reals in groups of four
//   spinor H16    uint2   [rhs][6][V] + float [rhs][V]: four FP16 values
//                 (components 2k, 2k+1) per uint2, scaled so that the site's
//                 largest real maps to 2^15, then the site's scale factor
//                 (52 bytes per site; storage only, arithmetic in FP32)
//
// A packed Hermitian 6x6 block holds its 6 real diagonal entries followed by
// the 15 complex entries below the diagonal in row order
// (1,0),(2,0),(2,1),(3,0),...,(5,4).  Block 0 acts on spins 0,1 (gamma_5 =
// +1), block 1 on spins 2,3; the block index within a chirality is
// 3*(spin & 1) + colour.  The stored matrix includes the unit diagonal of
// the operator: A(x) = 1 + i kappa c_sw sum_{mu<nu} sigma_{mu nu} F_{mu nu}(x).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <vector>

#include "../../include/qcd.h"

#define QCD_CUDA_OK(call)                                                    \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      qcd_set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,              \
                    cudaGetErrorString(e_));                                 \
      return QCD_ERR_CUDA;                                                   \
    }                                                                        \
  } while (0)

#define QCD_TRY(call)                                                        \
  do {                                                                       \
    qcd_status s_ = (call);                                                  \
    if (s_ != QCD_OK) return s_;                                             \
  } while (0)

void qcd_set_error(const char* fmt, ...);

// --------------------------------------------------------------------------
// Geometry
// --------------------------------------------------------------------------
struct Geom {
  int L[4];        // extents indexed by direction mu: 0 = t, 1 = x, 2 = y, 3 = z
  int V;           // sites
  int stride[4];   // site-index stride of a unit step in direction mu
  int bc_t;        // +1 periodic, -1 antiperiodic in time
};

__host__ __device__ inline void site_coords(const Geom& g, int s, int c[4]) {
  c[1] = s % g.L[1];
  int r = s / g.L[1];
  c[2] = r % g.L[2];
  r /= g.L[2];
  c[3] = r % g.L[3];
  c[0] = r / g.L[3];
}

// neighbour of site s (coordinate c) one step forward / backward in mu
__host__ __device__ inline int site_fwd(const Geom& g, int s, const int c[4], int mu) {
  return (c[mu] == g.L[mu] - 1) ? s - (g.L[mu] - 1) * g.stride[mu] : s + g.stride[mu];
}
__host__ __device__ inline int site_bwd(const Geom& g, int s, const int c[4], int mu) {
  return (c[mu] == 0) ? s + (g.L[mu] - 1) * g.stride[mu] : s - g.stride[mu];
}

// --------------------------------------------------------------------------
// Complex arithmetic on (re, im) pairs of a real type R
// --------------------------------------------------------------------------
template <typename R>
struct Cplx {
  R re, im;
};

template <typename R>
__host__ __device__ inline Cplx<R> cmk(R a, R b) { Cplx<R> z; z.re = a; z.im = b; return z; }
template <typename R>
__host__ __device__ inline Cplx<R> operator+(Cplx<R> a, Cplx<R> b) { return cmk(a.re + b.re, a.im + b.im); }
template <typename R>
__host__ __device__ inline Cplx<R> operator-(Cplx<R> a, Cplx<R> b) { return cmk(a.re - b.re, a.im - b.im); }
template <typename R>
__host__ __device__ inline Cplx<R> operator-(Cplx<R> a) { return cmk(-a.re, -a.im); }
template <typename R>
__host__ __device__ inline Cplx<R> operator*(Cplx<R> a, Cplx<R> b) {
  return cmk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R>
__host__ __device__ inline Cplx<R> operator*(R a, Cplx<R> b) { return cmk(a * b.re, a * b.im); }
template <typename R>
__host__ __device__ inline Cplx<R> conj(Cplx<R> a) { return cmk(a.re, -a.im); }
// conj(a) * b
template <typename R>
__host__ __device__ inline Cplx<R> cdot(Cplx<R> a, Cplx<R> b) {
  return cmk(a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re);
}
// Multiply-accumulate in fused steps (two roundings per real part instead of
// a product, a difference and a sum): acc += a * b, acc += conj(a) * b.
template <typename R>
__host__ __device__ inline R rfma(R a, R b, R c);
template <>
__host__ __device__ inline float rfma<float>(float a, float b, float c) { return fmaf(a, b, c); }
template <>
__host__ __device__ inline double rfma<double>(double a, double b, double c) { return fma(a, b, c); }
template <typename R>
__host__ __device__ inline void cmac(Cplx<R>& acc, Cplx<R> a, Cplx<R> b) {
  acc.re = rfma(a.re, b.re, acc.re);
  acc.re = rfma(-a.im, b.im, acc.re);
  acc.im = rfma(a.re, b.im, acc.im);
  acc.im = rfma(a.im, b.re, acc.im);
}
template <typename R>
__host__ __device__ inline void cmac_conj(Cplx<R>& acc, Cplx<R> a, Cplx<R> b) {
  acc.re = rfma(a.re, b.re, acc.re);
  acc.re = rfma(a.im, b.im, acc.re);
  acc.im = rfma(a.re, b.im, acc.im);
  acc.im = rfma(-a.im, b.re, acc.im);
}
// i * a, -i * a
template <typename R>
__host__ __device__ inline Cplx<R> mul_i(Cplx<R> a) { return cmk(-a.im, a.re); }
template <typename R>
__host__ __device__ inline Cplx<R> mul_mi(Cplx<R> a) { return cmk(a.im, -a.re); }

template <typename R>
struct Spinor {
  Cplx<R> c[12];   // 3*spin + colour
};
template <typename R>
struct HalfSpinor {
  Cplx<R> c[6];    // 3*s + colour, s = 0, 1
};
template <typename R>
struct SU3 {
  Cplx<R> m[3][3];
};

// --------------------------------------------------------------------------
// Spin projection in the chiral basis.  gamma_mu = [[0, e_mu], [e_mu^+, 0]]
// with e_0 = -1, e_k = -i sigma_k, so (1 -+ gamma_mu) psi = [h; -+ e_mu^+ h]
// with h = psi_up -+ e_mu psi_dn.  SIGN = -1 builds the (1 - gamma_mu)
// projection, SIGN = +1 the (1 + gamma_mu) projection.
// --------------------------------------------------------------------------
// w = e_mu v for a 2-spinor (per colour), e_0 = -1, e_k = -i sigma_k
template <int MU, typename R>
__host__ __device__ inline void e_mul(const Cplx<R> v0, const Cplx<R> v1, Cplx<R>& w0, Cplx<R>& w1) {
  if (MU == 0) { w0 = -v0; w1 = -v1; }
  if (MU == 1) { w0 = mul_mi(v1); w1 = mul_mi(v0); }          // -i sigma_1
  if (MU == 2) { w0 = -v1; w1 = v0; }                          // -i sigma_2 = [[0,-1],[1,0]]
  if (MU == 3) { w0 = mul_mi(v0); w1 = mul_i(v1); }            // -i sigma_3
}
// w = e_mu^+ v, e_0^+ = -1, e_k^+ = i sigma_k
template <int MU, typename R>
__host__ __device__ inline void edag_mul(const Cplx<R> v0, const Cplx<R> v1, Cplx<R>& w0, Cplx<R>& w1) {
  if (MU == 0) { w0 = -v0; w1 = -v1; }
  if (MU == 1) { w0 = mul_i(v1); w1 = mul_i(v0); }            // i sigma_1
  if (MU == 2) { w0 = v1; w1 = -v0; }                          // i sigma_2 = [[0,1],[-1,0]]
  if (MU == 3) { w0 = mul_i(v0); w1 = mul_mi(v1); }            // i sigma_3
}

template <int MU, int SIGN, typename R>
__host__ __device__ inline HalfSpinor<R> project(const Spinor<R>& p) {
  HalfSpinor<R> h;
#pragma unroll
  for (int a = 0; a < 3; a++) {
    Cplx<R> w0, w1;
    e_mul<MU>(p.c[6 + a], p.c[9 + a], w0, w1);
    if (SIGN < 0) { h.c[a] = p.c[a] - w0; h.c[3 + a] = p.c[3 + a] - w1; }
    else          { h.c[a] = p.c[a] + w0; h.c[3 + a] = p.c[3 + a] + w1; }
  }
  return h;
}

// out += scale * (1 SIGN gamma_mu)-reconstruction of h
template <int MU, int SIGN, typename R>
__host__ __device__ inline void accum_recon(Spinor<R>& out, const HalfSpinor<R>& h, R scale) {
#pragma unroll
  for (int a = 0; a < 3; a++) {
    Cplx<R> w0, w1;
    edag_mul<MU>(h.c[a], h.c[3 + a], w0, w1);
    out.c[a] = out.c[a] + scale * h.c[a];
    out.c[3 + a] = out.c[3 + a] + scale * h.c[3 + a];
    if (SIGN < 0) { out.c[6 + a] = out.c[6 + a] - scale * w0; out.c[9 + a] = out.c[9 + a] - scale * w1; }
    else          { out.c[6 + a] = out.c[6 + a] + scale * w0; out.c[9 + a] = out.c[9 + a] + scale * w1; }
  }
}

template <typename R>
__host__ __device__ inline HalfSpinor<R> su3_mul(const SU3<R>& U, const HalfSpinor<R>& h) {
  HalfSpinor<R> o;
#pragma unroll
  for (int s = 0; s < 2; s++)
#pragma unroll
    for (int a = 0; a < 3; a++) {
      Cplx<R> acc = U.m[a][0] * h.c[3 * s];
      cmac(acc, U.m[a][1], h.c[3 * s + 1]);
      cmac(acc, U.m[a][2], h.c[3 * s + 2]);
      o.c[3 * s + a] = acc;
    }
  return o;
}
template <typename R>
__host__ __device__ inline HalfSpinor<R> su3_dag_mul(const SU3<R>& U, const HalfSpinor<R>& h) {
  HalfSpinor<R> o;
#pragma unroll
  for (int s = 0; s < 2; s++)
#pragma unroll
    for (int a = 0; a < 3; a++) {
      Cplx<R> acc = cdot(U.m[0][a], h.c[3 * s]);
      cmac_conj(acc, U.m[1][a], h.c[3 * s + 1]);
      cmac_conj(acc, U.m[2][a], h.c[3 * s + 2]);
      o.c[3 * s + a] = acc;
    }
  return o;
}

// --------------------------------------------------------------------------
// Field access by precision.  Each precision has a storage struct with
// load/store for spinors, links and the clover term.
// --------------------------------------------------------------------------
struct FieldsD {   // FP64
  using R = double;
  static __device__ inline Spinor<double> load_spinor(const void* base, int V, int s) {
    const double2* p = (const double2*)base;
    Spinor<double> o;
#pragma unroll
    for (int c = 0; c < 12; c++) { double2 v = __ldg(p + (size_t)c * V + s); o.c[c] = cmk(v.x, v.y); }
    return o;
  }
  static __device__ inline void store_spinor(void* base, int V, int s, const Spinor<double>& o) {
    double2* p = (double2*)base;
#pragma unroll
    for (int c = 0; c < 12; c++) p[(size_t)c * V + s] = make_double2(o.c[c].re, o.c[c].im);
  }
  static __device__ inline SU3<double> load_link(const void* base, int V, int mu, int s) {
    const double2* p = (const double2*)base + (size_t)mu * 9 * V;
    SU3<double> U;
#pragma unroll
    for (int k = 0; k < 9; k++) { double2 v = __ldg(p + (size_t)k * V + s); U.m[k / 3][k % 3] = cmk(v.x, v.y); }
    return U;
  }
  // the 36 reals of chirality block b (0 or 1)
  static __device__ inline void load_clover_block(const void* base, int V, int s, int b, double (&cl)[36]) {
    const double2* p = (const double2*)base + (size_t)18 * b * V;
#pragma unroll
    for (int k = 0; k < 18; k++) { double2 v = __ldg(p + (size_t)k * V + s); cl[2 * k] = v.x; cl[2 * k + 1] = v.y; }
  }
  static constexpr size_t spinor_bytes = 192, link_bytes = 144, clover_bytes = 576;
};

struct FieldsF {   // FP32
  using R = float;
  static __device__ inline Spinor<float> load_spinor(const void* base, int V, int s) {
    const float4* p = (const float4*)base;
    Spinor<float> o;
#pragma unroll
    for (int k = 0; k < 6; k++) {
      float4 v = __ldg(p + (size_t)k * V + s);
      o.c[2 * k] = cmk(v.x, v.y);
      o.c[2 * k + 1] = cmk(v.z, v.w);
    }
    return o;
  }
  static __device__ inline void store_spinor(void* base, int V, int s, const Spinor<float>& o) {
    float4* p = (float4*)base;
#pragma unroll
    for (int k = 0; k < 6; k++)
      p[(size_t)k * V + s] = make_float4(o.c[2 * k].re, o.c[2 * k].im, o.c[2 * k + 1].re, o.c[2 * k + 1].im);
  }
  static __device__ inline SU3<float> load_link(const void* base, int V, int mu, int s) {
    const float4* p = (const float4*)base + (size_t)mu * 3 * V;
    float4 a = __ldg(p + s), b = __ldg(p + (size_t)V + s), c = __ldg(p + 2 * (size_t)V + s);
    SU3<float> U;
    U.m[0][0] = cmk(a.x, a.y); U.m[0][1] = cmk(a.z, a.w); U.m[0][2] = cmk(b.x, b.y);
    U.m[1][0] = cmk(b.z, b.w); U.m[1][1] = cmk(c.x, c.y); U.m[1][2] = cmk(c.z, c.w);
    // row 2 = conj(row0 x row1)
    U.m[2][0] = conj(U.m[0][1] * U.m[1][2] - U.m[0][2] * U.m[1][1]);
    U.m[2][1] = conj(U.m[0][2] * U.m[1][0] - U.m[0][0] * U.m[1][2]);
    U.m[2][2] = conj(U.m[0][0] * U.m[1][1] - U.m[0][1] * U.m[1][0]);
    return U;
  }
  static __device__ inline void load_clover_block(const void* base, int V, int s, int b, float (&cl)[36]) {
    const float4* p = (const float4*)base + (size_t)9 * b * V;
#pragma unroll
    for (int k = 0; k < 9; k++) {
      float4 v = __ldg(p + (size_t)k * V + s);
      cl[4 * k] = v.x; cl[4 * k + 1] = v.y; cl[4 * k + 2] = v.z; cl[4 * k + 3] = v.w;
    }
  }
  static constexpr size_t spinor_bytes = 96, link_bytes = 48, clover_bytes = 288;
};

// Internal precision code of the FP16 + per-site scale storage (Krylov images
// chi_k of the sloppy solves); never accepted at the C-ABI.
constexpr int QCD_PREC_H16 = 2;

__device__ inline unsigned h2_bits(__half2 h) { return *reinterpret_cast<unsigned*>(&h); }
__device__ inline __half2 bits_h2(unsigned u) { return *reinterpret_cast<__half2*>(&u); }

struct FieldsH {   // FP16 spinor storage with one FP32 scale per site
  using R = float;
  static constexpr float kTop = 32768.f;   // the site's largest |real| is stored as 2^15
  static constexpr float kTiny = 1e-30f;
  static constexpr size_t spinor_bytes = 52;
  static __device__ inline const float* scale_ptr(const void* base, int V) {
    return (const float*)((const uint2*)base + 6 * (size_t)V);
  }
  // site value = scale * (FP16 word); encode and decode are the exact steps
  // of a store and a later load, so a kernel can round in registers
  static __device__ inline void encode(const Spinor<float>& o, uint2 (&w)[6], float& sc) {
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < 12; k++) m = fmaxf(m, fmaxf(fabsf(o.c[k].re), fabsf(o.c[k].im)));
    // sites whose largest |real| is below kTiny are stored as zero: 2^15 / m
    // would overflow FP32 below about 1e-34, and such entries are negligible
    // against any vector the solver normalises
    const float f = m > kTiny ? kTop / m : 0.f;
#pragma unroll
    for (int k = 0; k < 6; k++) {
      const __half2 a = __floats2half2_rn(f * o.c[2 * k].re, f * o.c[2 * k].im);
      const __half2 b = __floats2half2_rn(f * o.c[2 * k + 1].re, f * o.c[2 * k + 1].im);
      w[k] = make_uint2(h2_bits(a), h2_bits(b));
    }
    sc = f > 0.f ? m / kTop : 0.f;
  }
  static __device__ inline Spinor<float> decode(const uint2 (&w)[6], float sc) {
    Spinor<float> o;
#pragma unroll
    for (int k = 0; k < 6; k++) {
      const float2 a = __half22float2(bits_h2(w[k].x)), b = __half22float2(bits_h2(w[k].y));
      o.c[2 * k] = cmk(sc * a.x, sc * a.y);
      o.c[2 * k + 1] = cmk(sc * b.x, sc * b.y);
    }
    return o;
  }
  static __device__ inline void load_words(const void* base, int V, int s, uint2 (&w)[6], float& sc) {
    const uint2* p = (const uint2*)base;
    sc = __ldg(scale_ptr(base, V) + s);
#pragma unroll
    for (int k = 0; k < 6; k++) w[k] = __ldg(p + (size_t)k * V + s);
  }
  static __device__ inline Spinor<float> load_spinor(const void* base, int V, int s) {
    uint2 w[6];
    float sc;
    load_words(base, V, s, w, sc);
    return decode(w, sc);
  }
  static __device__ inline void store_spinor(void* base, int V, int s, const Spinor<float>& o) {
    uint2 w[6];
    float sc;
    encode(o, w, sc);
    uint2* p = (uint2*)base;
#pragma unroll
    for (int k = 0; k < 6; k++) p[(size_t)k * V + s] = w[k];
    ((float*)scale_ptr(base, V))[s] = sc;
  }
};

// Apply one packed Hermitian 6x6 block (36 reals starting at cl[k0]) to v.
template <typename R>
__host__ __device__ inline void clover_block_apply(const R* cl, int k0, const Cplx<R>* v, Cplx<R>* out) {
#pragma unroll
  for (int i = 0; i < 6; i++) out[i] = cl[k0 + i] * v[i];
  int k = k0 + 6;
#pragma unroll
  for (int i = 1; i < 6; i++) {
#pragma unroll
    for (int j = 0; j < i; j++) {
      Cplx<R> h = cmk(cl[k], cl[k + 1]);
      k += 2;
      cmac(out[i], h, v[j]);
      cmac_conj(out[j], h, v[i]);
    }
  }
}

// A(x) psi(x): the site-diagonal part of the operator (unit + clover term),
// one chirality block at a time
template <typename F>
__device__ inline Spinor<typename F::R> clover_apply(const void* clv, int V, int s, const Spinor<typename F::R>& p) {
  Spinor<typename F::R> o;
#pragma unroll
  for (int b = 0; b < 2; b++) {
    typename F::R cl[36];
    F::load_clover_block(clv, V, s, b, cl);
    clover_block_apply(cl, 0, &p.c[6 * b], &o.c[6 * b]);
  }
  return o;
}

// --------------------------------------------------------------------------
// The context
// --------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

qcd_status devbuf_ensure(DevBuf& b, size_t bytes);
void devbuf_free(DevBuf& b);

// kernel families of the timing records (qcd_profile_read)
enum ProfFam { FAM_DSLASH_D, FAM_DSLASH_F, FAM_SAP_D, FAM_SAP_F, FAM_BLAS, FAM_LAYOUT, FAM_CONTRACT, FAM_DFL, FAM_N };

struct ProfRec {
  int fam, kernels;
  cudaEvent_t a, b;
  double bytes, flops;
};

struct SapGraph {
  const void *rho_src, *rho, *psi, *delta, *gauge, *clover;
  const int* mask;
  int nrhs, ncy, nmr, accumulate, half, prec, block[4];
  double kappa;
  cudaGraphExec_t exec;
};

struct qcd_ctx {
  int prof_on = 0;
  int prof_suspend = 0;          // > 0 while a stream is being captured
  std::vector<SapGraph> sap_graphs;
  std::vector<ProfRec> prof;
  std::vector<cudaEvent_t> evpool;
  Geom g;
  int dims[4];     // T, X, Y, Z as given by the caller
  cudaStream_t stream;
  double kappa = 0, csw = 0;
  int have_gauge = 0;
  qcd_solver_params params;
  // fields
  DevBuf gaugeD, gaugeF, cloverD, cloverF;
  // FP16 copies for the sloppy SAP block solves (layout.cu): links as the nine
  // (re, im) entries of the full matrix (third row reconstructed in FP32 from
  // the FP32 rows, then rounded), [4][V] uint4 of entries 0-3, [4][V] uint4 of
  // entries 4-7, [4][V] uint32 of entry 8 (36 B per link); clover as
  // [9][V] uint4 of eight FP16 reals (144 B per site)
  DevBuf gaugeH, cloverH;
  // workspaces (grown on demand, kept until destroy)
  DevBuf wsD[8];      // FP64 spinors (nrhs each)
  DevBuf wsF[8];      // FP32 spinors
  DevBuf basisF;      // Krylov basis phi/chi (FP32)
  DevBuf basisD;      // Krylov basis for the all-FP64 policy
  DevBuf red;         // reduction partials
  DevBuf scal;        // device scalars of the solver
  DevBuf contract;    // per-site contraction values
  DevBuf stage;       // staging for host <-> device copies
  DevBuf guess;       // sloppy solutions reused as initial guesses of exact solves
  DevBuf small;       // small per-call arrays (source sites, dot products), kept between calls
  double* host_scal = nullptr;   // pinned mirror of scalars
  size_t host_scal_bytes = 0;
  void* dfl = nullptr;           // deflation state (dfl.cu)
  // smeared sources and sinks (smear.cu): APE-smeared links (FP64, internal
  // gauge layout; time links copied), Gaussian kernel parameters, scratch
  DevBuf gaugeS;
  int have_smeared_links = 0;
  double smear_kappa = 0;
  int smear_n = 0;               // 0: point sources and sinks
  DevBuf smearbuf[2];
};

// Brackets the launches issued in its scope with CUDA events when profiling
// is enabled; bytes and flops are the algorithmic counts of those launches.
struct ProfScope {
  qcd_ctx* c;
  int idx;
  ProfScope(qcd_ctx* c, int fam, double bytes, double flops, int kernels = 1);
  ~ProfScope();
};

// --------------------------------------------------------------------------
// Internal entry points shared between the .cu files
// --------------------------------------------------------------------------
qcd_status layout_gauge_import(qcd_ctx* c, const double* U_dev);
qcd_status layout_clover_build(qcd_ctx* c);
// canonical [rhs][V][4][3] complex FP64 <-> internal spinor of precision prec (0 FP64, 1 FP32)
qcd_status layout_spinor_import(qcd_ctx* c, const double* in, void* out, int prec, int nrhs);
qcd_status layout_spinor_export(qcd_ctx* c, const void* in, double* out, int prec, int nrhs);
qcd_status clover_export(qcd_ctx* c, double* out_dev);

// out = D in (or D^+), internal layout, precision prec; mask may be null,
// nactive = number of unmasked right-hand sides (for the timing records);
// out_prec = QCD_PREC_H16 stores an FP32 operator's output as FP16 + scale
qcd_status dslash_apply(qcd_ctx* c, const void* in, void* out, int prec, int nrhs, int dagger, const int* mask,
                        int nactive, int out_prec = -1);

// reductions / vector ops (internal layouts; n = 12 V complex per rhs)
qcd_status blas_norm2(qcd_ctx* c, const void* x, int prec, int nrhs, double* out_dev, const int* mask);
qcd_status blas_dot(qcd_ctx* c, const void* x, int precx, const void* y, int precy, int nrhs, double* out_dev,
                    const int* mask);
qcd_status blas_convert(qcd_ctx* c, const void* in, int pin, void* out, int pout, int nrhs, const int* mask);
// y_r += sign * sum_{j<nx} coef[j*nrhs + r] x_{j,r}; x_j at xbase + j*xstride bytes
qcd_status blas_multi_caxpy(qcd_ctx* c, void* y, int py, const void* xbase, int px, int nx, size_t xstride,
                            const double* coef_dev, double sign, int nrhs, const int* mask);
qcd_status blas_scale(qcd_ctx* c, void* x, int px, const double* sc_dev, int nrhs, const int* mask);
// fused Gram-Schmidt step of the GCR cycle (chi_j at chi + j*jstride bytes, j <= k)
qcd_status blas_gs_dots(qcd_ctx* c, const void* chi, int prec, size_t jstride, int k, int nrhs, double* dots_dev,
                        const int* mask, int nactive);
qcd_status blas_gs_orth(qcd_ctx* c, void* chi, int prec, size_t jstride, int k, const double* dots_dev,
                        const void* rho, int prho, int nrhs, double* n2c_dev, const int* mask, int nactive);
// chi_k *= inv; rho -= ck chi_k; chi_k in precision pchi (F64, F32 or H16),
// rho in the inner precision prho
qcd_status blas_gs_finish_inner(qcd_ctx* c, void* chik, int pchi, const double* inv_dev, const double* ck_dev,
                                void* rho, int prho, int nrhs, double* rn2_dev, const int* mask, int nactive);
// out = x - y
qcd_status blas_xmy(qcd_ctx* c, const void* x, const void* y, void* out, int prec, int nrhs, const int* mask);

// SAP preconditioner: psi = M_SAP rho (rho is overwritten), precision prec
// psi = M_SAP rho_src (accumulate != 0: psi += M_SAP rho_src); rho is the SAP's
// working residual (overwritten); rho_src = nullptr means rho itself
qcd_status sap_apply(qcd_ctx* c, void* rho, void* psi, void* delta, int prec, int nrhs, const int* mask,
                     int nactive, int accumulate = 0, const void* rho_src = nullptr);

// deflation (dfl.cu)
qcd_status dfl_setup(qcd_ctx* c, const double* init_dev, int ns, int n_inv);
qcd_status dfl_low_mode(qcd_ctx* c, const void* rho, void* x, int n, const int* mask, int nactive, int m);
qcd_status dfl_little_host(qcd_ctx* c, const double* in, double* out, int n, int mode, int m);
void dfl_free(qcd_ctx* c);
int dfl_ready(qcd_ctx* c);
int dfl_ns(qcd_ctx* c);
int dfl_nblk(qcd_ctx* c);
void* dfl_phi(qcd_ctx* c);
void* dfl_little(qcd_ctx* c);

size_t spinor_bytes(const qcd_ctx* c, int prec);

// Gaussian smearing (smear.cu) of nrhs FP64 internal spinors in place with
// the context's smeared links and parameters (a no-op when smear_n is 0)
qcd_status smear_fields(qcd_ctx* c, void* fields, int nrhs);
