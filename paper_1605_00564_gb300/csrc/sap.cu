// Schwarz alternating procedure (Sec. 2.2).
//
// The lattice is split into blocks of extent b = (bt, bx, by, bz) coloured
// as a checkerboard (colour = parity of the block coordinates); D_Omega is the
// operator restricted to the black blocks with the hops that leave a block
// dropped (Dirichlet), D_dOmega* the hops from Omega into the white blocks.
// n_cy cycles, each visiting all black then all white blocks, applied to
// psi = 0 give M_SAP = K sum_{nu<n_cy} (1 - D K)^nu.
//
// Residual form of a half-cycle on colour c (rho = eta - D psi):
//   on every block L of colour c:  x = approx D_L^-1 rho_L (n_mr MR steps from 0),
//                                   psi_L += x,  rho_L = rho_L - D_L x,  delta_L = x
//   on the neighbouring sites y of the other colour: rho(y) -= (D delta)(y)
// The last line touches only blocks of the other colour, which are the next
// half-cycle's blocks, so it is applied there as a gather at the start of the
// next sweep: each site at a block face adds kappa * hop(delta) from the
// neighbouring block (delta of the previous half-cycle).  No two CTAs write
// the same word, so the result does not depend on scheduling.
//
// One CTA per block and right-hand side, one thread per block site; the
// block's residual lives in shared memory across the MR steps, the solution
// increment x in registers.
#include <string.h>

#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "qcd_internal.cuh"

namespace {

struct SapGeom {
  int b[4];     // block extents by direction (t, x, y, z)
  int nb[4];    // blocks per direction
  int lst[4];   // local stride of direction mu inside a block
  int vb;       // block volume
};

template <typename R>
__device__ inline Spinor<R> smem_load(const Cplx<R>* r_s, int vb, int l) {
  Spinor<R> o;
#pragma unroll
  for (int k = 0; k < 12; k++) o.c[k] = r_s[k * vb + l];
  return o;
}
template <typename R>
__device__ inline void smem_store(Cplx<R>* r_s, int vb, int l, const Spinor<R>& v) {
#pragma unroll
  for (int k = 0; k < 12; k++) r_s[k * vb + l] = v.c[k];
}

// p += scale * (hops of the block operator inside the block, applied to r_s)
template <typename F, int MU>
__device__ inline void block_hop(Spinor<typename F::R>& p, const Cplx<typename F::R>* r_s, const SapGeom& sg,
                                 const void* gauge, const Geom& g, int s, int l, const int lc[4],
                                 typename F::R scale) {
  using R = typename F::R;
  if (lc[MU] < sg.b[MU] - 1) {
    HalfSpinor<R> h = project<MU, -1>(smem_load(r_s, sg.vb, l + sg.lst[MU]));
    h = su3_mul(F::load_link(gauge, g.V, MU, s), h);
    accum_recon<MU, -1>(p, h, scale);
  }
  if (lc[MU] > 0) {
    HalfSpinor<R> h = project<MU, +1>(smem_load(r_s, sg.vb, l - sg.lst[MU]));
    h = su3_dag_mul(F::load_link(gauge, g.V, MU, s - g.stride[MU]), h);
    accum_recon<MU, +1>(p, h, scale);
  }
}

// r += scale * (hops from delta on the neighbouring blocks, across this block's faces)
template <typename F, int MU>
__device__ inline void face_hop(Spinor<typename F::R>& hop, const char* delta, const SapGeom& sg, const void* gauge,
                                const Geom& g, int s, const int c[4], const int lc[4], typename F::R scale) {
  using R = typename F::R;
  if (lc[MU] == sg.b[MU] - 1) {
    int sf = site_fwd(g, s, c, MU);
    R sign = (MU == 0 && c[0] == g.L[0] - 1) ? (R)g.bc_t * scale : scale;
    HalfSpinor<R> h = project<MU, -1>(F::load_spinor(delta, g.V, sf));
    h = su3_mul(F::load_link(gauge, g.V, MU, s), h);
    accum_recon<MU, -1>(hop, h, sign);
  }
  if (lc[MU] == 0) {
    int sb = site_bwd(g, s, c, MU);
    R sign = (MU == 0 && c[0] == 0) ? (R)g.bc_t * scale : scale;
    HalfSpinor<R> h = project<MU, +1>(F::load_spinor(delta, g.V, sb));
    h = su3_dag_mul(F::load_link(gauge, g.V, MU, sb), h);
    accum_recon<MU, +1>(hop, h, sign);
  }
}

template <typename R>
__device__ inline R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename F, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) k_sap_sweep(const char* __restrict__ rho_src, char* __restrict__ rho,
                                                          char* __restrict__ psi, char* __restrict__ delta,
                            const void* __restrict__ gauge, const void* __restrict__ clover, Geom g, SapGeom sg,
                            int colour, int gather, int psi_init, typename F::R kappa, int nmr, int nrhs,
                            const int* mask) {
  using R = typename F::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cplx<R>* r_s = (Cplx<R>*)smem_raw;
  __shared__ R red[3][32];

  // the RHS index runs fastest over the grid: the CTAs of one block (all RHS)
  // are resident together and share its links and clover term through L2
  const int rhs = blockIdx.x % nrhs;
  const int blk = blockIdx.x / nrhs;
  if (mask && !mask[rhs]) return;
  const size_t off = (size_t)rhs * F::spinor_bytes * g.V;
  rho_src += off;
  rho += off;
  psi += off;
  delta += off;

  // which block: the blk-th block of this colour
  const int nbx2 = sg.nb[1] >> 1;
  int q = blk / nbx2;
  const int j = blk - q * nbx2;
  const int by = q % sg.nb[2];
  q /= sg.nb[2];
  const int bz = q % sg.nb[3];
  const int bt = q / sg.nb[3];
  const int bx = 2 * j + ((colour + bt + bz + by) & 1);

  const int l = threadIdx.x;
  int lc[4], c[4];
  {
    int r = l;
    lc[1] = r % sg.b[1]; r /= sg.b[1];
    lc[2] = r % sg.b[2]; r /= sg.b[2];
    lc[3] = r % sg.b[3];
    lc[0] = r / sg.b[3];
  }
  c[0] = bt * sg.b[0] + lc[0];
  c[1] = bx * sg.b[1] + lc[1];
  c[2] = by * sg.b[2] + lc[2];
  c[3] = bz * sg.b[3] + lc[3];
  const int s = ((c[0] * g.L[3] + c[3]) * g.L[2] + c[2]) * g.L[1] + c[1];

  // pending boundary update from the previous half-cycle
  Spinor<R> r = F::load_spinor(rho_src, g.V, s);
  if (gather) {
    face_hop<F, 0>(r, delta, sg, gauge, g, s, c, lc, kappa);
    face_hop<F, 1>(r, delta, sg, gauge, g, s, c, lc, kappa);
    face_hop<F, 2>(r, delta, sg, gauge, g, s, c, lc, kappa);
    face_hop<F, 3>(r, delta, sg, gauge, g, s, c, lc, kappa);
  }
  smem_store(r_s, sg.vb, l, r);

  Spinor<R> x;
#pragma unroll
  for (int k = 0; k < 12; k++) x.c[k] = cmk((R)0, (R)0);

  const int warp = l >> 5, lane = l & 31, nw = (sg.vb + 31) >> 5;
  for (int step = 0; step < nmr; step++) {
    __syncthreads();
    // p = D_L r
    Spinor<R> p = clover_apply<F>(clover, g.V, s, r);
    block_hop<F, 0>(p, r_s, sg, gauge, g, s, l, lc, -kappa);
    block_hop<F, 1>(p, r_s, sg, gauge, g, s, l, lc, -kappa);
    block_hop<F, 2>(p, r_s, sg, gauge, g, s, l, lc, -kappa);
    block_hop<F, 3>(p, r_s, sg, gauge, g, s, l, lc, -kappa);
    // alpha = (p, r) / (p, p) over the block
    Cplx<R> pr = cmk((R)0, (R)0);
    R pp = 0;
#pragma unroll
    for (int k = 0; k < 12; k++) {
      cmac_conj(pr, p.c[k], r.c[k]);
      pp = rfma(p.c[k].re, p.c[k].re, pp);
      pp = rfma(p.c[k].im, p.c[k].im, pp);
    }
    R pr_re = pr.re, pr_im = pr.im;
    pr_re = warp_sum(pr_re);
    pr_im = warp_sum(pr_im);
    pp = warp_sum(pp);
    if (lane == 0) {
      red[0][warp] = pr_re;
      red[1][warp] = pr_im;
      red[2][warp] = pp;
    }
    __syncthreads();
    R a_re = 0, a_im = 0, n2 = 0;
    for (int w = 0; w < nw; w++) {
      a_re += red[0][w];
      a_im += red[1][w];
      n2 += red[2][w];
    }
    Cplx<R> alpha = n2 > (R)0 ? cmk(a_re / n2, a_im / n2) : cmk((R)0, (R)0);
    const Cplx<R> malpha = -alpha;
#pragma unroll
    for (int k = 0; k < 12; k++) {
      cmac(x.c[k], alpha, r.c[k]);
      cmac(r.c[k], malpha, p.c[k]);
    }
    __syncthreads();
    smem_store(r_s, sg.vb, l, r);
  }

  if (psi_init) {
    F::store_spinor(psi, g.V, s, x);
  } else {
    Spinor<R> y = F::load_spinor(psi, g.V, s);
#pragma unroll
    for (int k = 0; k < 12; k++) y.c[k] = y.c[k] + x.c[k];
    F::store_spinor(psi, g.V, s, y);
  }
  F::store_spinor(rho, g.V, s, r);
  F::store_spinor(delta, g.V, s, x);
}

// ---------------------------------------------------------------------------
// Shared-memory-resident variant (FP32 arithmetic).  The block's links (two
// rows each) and clover term are staged in shared memory once per sweep, so
// the n_mr MR steps read only shared memory.  S selects the storage of the
// staged copies: float (exact single precision) or __half (16-bit copies of
// links and clover, half the shared memory, two CTAs per SM; the
// preconditioner is then a slightly different operator, which the flexible
// outer GCR tolerates).
// ---------------------------------------------------------------------------
template <typename S>
struct Stage;
template <>
struct Stage<float> {
  using W = float4;   // four reals
  using C = float2;   // one complex
  static __device__ inline W put(float4 v) { return v; }
  static __device__ inline float4 get(W w) { return w; }
  static __device__ inline C putc(Cplx<float> z) { return make_float2(z.re, z.im); }
  static __device__ inline Cplx<float> getc(C w) { return cmk(w.x, w.y); }
};
template <>
struct Stage<__half> {
  using W = uint2;
  static __device__ inline W put(float4 v) {
    __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
    W w;
    w.x = *reinterpret_cast<unsigned*>(&a);
    w.y = *reinterpret_cast<unsigned*>(&b);
    return w;
  }
  static __device__ inline float4 get(W w) {
    float2 a = __half22float2(*reinterpret_cast<__half2*>(&w.x));
    float2 b = __half22float2(*reinterpret_cast<__half2*>(&w.y));
    return make_float4(a.x, a.y, b.x, b.y);
  }
  using C = __half2;
  static __device__ inline C putc(Cplx<float> z) { return __floats2half2_rn(z.re, z.im); }
  static __device__ inline Cplx<float> getc(C w) {
    float2 a = __half22float2(w);
    return cmk(a.x, a.y);
  }
};

// Storage of the block residual shared between neighbouring threads:
// FP32 complex, or bf16 pairs (FP32 exponent range, 8-bit mantissa; each
// thread keeps its own residual in FP32 registers, only the neighbours'
// contributions to p = D_L r see the rounding).
template <bool BF>
struct RStore;
template <>
struct RStore<false> {
  using T = Cplx<float>;
  static __device__ inline T put(Cplx<float> z) { return z; }
  static __device__ inline Cplx<float> get(T t) { return t; }
};
template <>
struct RStore<true> {
  using T = __nv_bfloat162;
  static __device__ inline T put(Cplx<float> z) { return __floats2bfloat162_rn(z.re, z.im); }
  static __device__ inline Cplx<float> get(T t) {
    float2 f = __bfloat1622float2(t);
    return cmk(f.x, f.y);
  }
};
// FP32: 16-byte records, word q of site l at ((float4*)r_s)[q * vb + l] holding
// components 2q and 2q + 1 (one 128-bit load per two components); bf16: one
// 4-byte word per component at r_s[k * vb + l]
template <bool BF>
__device__ inline Spinor<float> rs_load(const typename RStore<BF>::T* r_s, int vb, int l) {
  Spinor<float> o;
  if (BF) {
#pragma unroll
    for (int k = 0; k < 12; k++) o.c[k] = RStore<BF>::get(r_s[k * vb + l]);
  } else {
    const float4* w = reinterpret_cast<const float4*>(r_s);
#pragma unroll
    for (int q = 0; q < 6; q++) {
      const float4 v = w[q * vb + l];
      o.c[2 * q] = cmk(v.x, v.y);
      o.c[2 * q + 1] = cmk(v.z, v.w);
    }
  }
  return o;
}
template <bool BF>
__device__ inline void rs_store(typename RStore<BF>::T* r_s, int vb, int l, const Spinor<float>& v) {
  if (BF) {
#pragma unroll
    for (int k = 0; k < 12; k++) r_s[k * vb + l] = RStore<BF>::put(v.c[k]);
  } else {
    float4* w = reinterpret_cast<float4*>(r_s);
#pragma unroll
    for (int q = 0; q < 6; q++)
      w[q * vb + l] = make_float4(v.c[2 * q].re, v.c[2 * q].im, v.c[2 * q + 1].re, v.c[2 * q + 1].im);
  }
}

// the full 3x3 link (staged with its third row already reconstructed)
template <typename S>
__device__ inline SU3<float> smem_link(const typename Stage<S>::C* lk, int vb, int mu, int l) {
  const typename Stage<S>::C* p = lk + (size_t)mu * 9 * vb;
  SU3<float> U;
#pragma unroll
  for (int k = 0; k < 9; k++) U.m[k / 3][k % 3] = Stage<S>::getc(p[(size_t)k * vb + l]);
  return U;
}

template <typename S>
__device__ inline Spinor<float> smem_clover_apply(const typename Stage<S>::W* cl, int vb, int l,
                                                  const Spinor<float>& p) {
  Spinor<float> o;
#pragma unroll
  for (int b = 0; b < 2; b++) {
    float c[36];
#pragma unroll
    for (int k = 0; k < 9; k++) {
      float4 v = Stage<S>::get(cl[(size_t)(9 * b + k) * vb + l]);
      c[4 * k] = v.x; c[4 * k + 1] = v.y; c[4 * k + 2] = v.z; c[4 * k + 3] = v.w;
    }
    clover_block_apply(c, 0, &p.c[6 * b], &o.c[6 * b]);
  }
  return o;
}

template <typename S, bool BF, int MU>
__device__ inline void smem_block_hop(Spinor<float>& p, const typename RStore<BF>::T* r_s,
                                      const typename Stage<S>::C* lk, const SapGeom& sg, int l, const int lc[4],
                                      float scale) {
  if (lc[MU] < sg.b[MU] - 1) {
    HalfSpinor<float> h = project<MU, -1>(rs_load<BF>(r_s, sg.vb, l + sg.lst[MU]));
    h = su3_mul(smem_link<S>(lk, sg.vb, MU, l), h);
    accum_recon<MU, -1>(p, h, scale);
  }
  if (lc[MU] > 0) {
    HalfSpinor<float> h = project<MU, +1>(rs_load<BF>(r_s, sg.vb, l - sg.lst[MU]));
    h = su3_dag_mul(smem_link<S>(lk, sg.vb, MU, l - sg.lst[MU]), h);
    accum_recon<MU, +1>(p, h, scale);
  }
}

// One direction of the boundary gather with the block residual in shared
// memory (FP32): every site on the +MU face and every site on the -MU face
// (disjoint sets for b_MU >= 2) receives the hop from the neighbouring block's
// delta.  One thread per face site, so all lanes of the busy warps work; the
// site's residual is read, updated and written back by that thread, in the
// same arithmetic as a per-site update.  co: the block's first site.
template <int MU>
__device__ inline void smem_gather_dir(Cplx<float>* r_s, const SapGeom& sg, const Geom& g, const char* delta,
                                       const float4* gauge, const int co[4], int l, float kappa) {
  const int nface = sg.vb / sg.b[MU];
  if (l >= 2 * nface) return;
  const bool fwd = l < nface;
  int t = fwd ? l : l - nface;
  int lc[4], c[4];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const int nu = (k + 1) & 3;   // x, y, z, then t
    if (nu == MU) {
      lc[nu] = fwd ? sg.b[MU] - 1 : 0;
    } else {
      lc[nu] = t % sg.b[nu];
      t /= sg.b[nu];
    }
  }
  const int ls = lc[0] * sg.lst[0] + lc[1] * sg.lst[1] + lc[2] * sg.lst[2] + lc[3] * sg.lst[3];
#pragma unroll
  for (int mu = 0; mu < 4; mu++) c[mu] = co[mu] + lc[mu];
  const int s = ((c[0] * g.L[3] + c[3]) * g.L[2] + c[2]) * g.L[1] + c[1];
  Spinor<float> r = rs_load<false>(r_s, sg.vb, ls);
  if (fwd) {
    const int sf = site_fwd(g, s, c, MU);
    const float sign = (MU == 0 && c[0] == g.L[0] - 1) ? (float)g.bc_t * kappa : kappa;
    HalfSpinor<float> h = project<MU, -1>(FieldsF::load_spinor(delta, g.V, sf));
    h = su3_mul(FieldsF::load_link(gauge, g.V, MU, s), h);
    accum_recon<MU, -1>(r, h, sign);
  } else {
    const int sb = site_bwd(g, s, c, MU);
    const float sign = (MU == 0 && c[0] == 0) ? (float)g.bc_t * kappa : kappa;
    HalfSpinor<float> h = project<MU, +1>(FieldsF::load_spinor(delta, g.V, sb));
    h = su3_dag_mul(FieldsF::load_link(gauge, g.V, MU, sb), h);
    accum_recon<MU, +1>(r, h, sign);
  }
  rs_store<false>(r_s, sg.vb, ls, r);
}

// B4 = true: the block is 4^4, known at compile time, so every shared-memory
// offset (component stride vb, neighbour strides) is an immediate.
template <typename S, bool BF, bool B4, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB)
    k_sap_sweep_smem(const char* __restrict__ rho_src, char* __restrict__ rho, char* __restrict__ psi,
                     char* __restrict__ delta,
                     const float4* __restrict__ gauge, const float4* __restrict__ clover,
                     const uint4* __restrict__ gaugeH, const uint4* __restrict__ cloverH, Geom g, SapGeom sg_in,
                     int colour, int gather, int psi_init, float kappa, int nmr, int nrhs, const int* mask) {
  SapGeom sg = sg_in;
  if (B4) {
    sg.b[0] = sg.b[1] = sg.b[2] = sg.b[3] = 4;
    sg.lst[1] = 1;
    sg.lst[2] = 4;
    sg.lst[3] = 16;
    sg.lst[0] = 64;
    sg.vb = 256;
  }
  using W = typename Stage<S>::W;
  using CW = typename Stage<S>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int vb = sg.vb;
  using RT = typename RStore<BF>::T;
  RT* r_s = (RT*)smem_raw;
  CW* lk_s = (CW*)(smem_raw + (size_t)12 * vb * sizeof(RT));              // [4][9][vb]
  W* cl_s = (W*)(lk_s + (size_t)36 * vb);                                 // [18][vb]
  __shared__ float4 red[32];   // per warp: (p, r) re, im, (p, p)

  const int rhs = blockIdx.x % nrhs;   // RHS fastest, as in k_sap_sweep
  const int blk = blockIdx.x / nrhs;
  if (mask && !mask[rhs]) return;
  const size_t off = (size_t)rhs * FieldsF::spinor_bytes * g.V;
  rho_src += off;
  rho += off;
  psi += off;
  delta += off;

  const int nbx2 = sg.nb[1] >> 1;
  int q = blk / nbx2;
  const int j = blk - q * nbx2;
  const int by = q % sg.nb[2];
  q /= sg.nb[2];
  const int bz = q % sg.nb[3];
  const int bt = q / sg.nb[3];
  const int bx = 2 * j + ((colour + bt + bz + by) & 1);

  const int l = threadIdx.x;
  int lc[4], c[4];
  {
    int r = l;
    lc[1] = r % sg.b[1]; r /= sg.b[1];
    lc[2] = r % sg.b[2]; r /= sg.b[2];
    lc[3] = r % sg.b[3];
    lc[0] = r / sg.b[3];
  }
  c[0] = bt * sg.b[0] + lc[0];
  c[1] = bx * sg.b[1] + lc[1];
  c[2] = by * sg.b[2] + lc[2];
  c[3] = bz * sg.b[3] + lc[3];
  const int s = ((c[0] * g.L[3] + c[3]) * g.L[2] + c[2]) * g.L[1] + c[1];

  // stage this site's four links (full 3x3) and its clover term: 16-bit
  // copies straight from their FP16 copies in HBM (rounded once at gauge
  // load, as the FP32 path rounds them here), FP32 copies from the FP32 fields
  if (std::is_same<S, __half>::value) {
    const uint4* gB = gaugeH + 4 * (size_t)g.V;
    const unsigned* gC = (const unsigned*)(gB + 4 * (size_t)g.V);
    unsigned* lw = (unsigned*)lk_s;
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
      const uint4 a = __ldg(gaugeH + (size_t)mu * g.V + s), b = __ldg(gB + (size_t)mu * g.V + s);
      const unsigned h8 = __ldg(gC + (size_t)mu * g.V + s);
      const unsigned w[9] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, h8};
#pragma unroll
      for (int k = 0; k < 9; k++) lw[(size_t)(9 * mu + k) * vb + l] = w[k];
    }
    uint2* cw = (uint2*)cl_s;
#pragma unroll
    for (int k = 0; k < 9; k++) {
      const uint4 v = __ldg(cloverH + (size_t)k * g.V + s);
      cw[(size_t)(2 * k) * vb + l] = make_uint2(v.x, v.y);
      cw[(size_t)(2 * k + 1) * vb + l] = make_uint2(v.z, v.w);
    }
  } else {
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
      SU3<float> U = FieldsF::load_link(gauge, g.V, mu, s);
#pragma unroll
      for (int k = 0; k < 9; k++) lk_s[(size_t)(9 * mu + k) * vb + l] = Stage<S>::putc(U.m[k / 3][k % 3]);
    }
#pragma unroll
    for (int k = 0; k < 18; k++) cl_s[(size_t)k * vb + l] = Stage<S>::put(__ldg(clover + (size_t)k * g.V + s));
  }

  Spinor<float> r = FieldsF::load_spinor(rho_src, g.V, s);
  if (BF) {
    // bf16 shared residual: the site's own residual stays FP32 in registers
    if (gather) {
      face_hop<FieldsF, 0>(r, delta, sg, gauge, g, s, c, lc, kappa);
      face_hop<FieldsF, 1>(r, delta, sg, gauge, g, s, c, lc, kappa);
      face_hop<FieldsF, 2>(r, delta, sg, gauge, g, s, c, lc, kappa);
      face_hop<FieldsF, 3>(r, delta, sg, gauge, g, s, c, lc, kappa);
    }
    rs_store<BF>(r_s, vb, l, r);
  } else {
    rs_store<BF>(r_s, vb, l, r);
    if (gather) {
      // boundary term in four rounds (one direction each, both faces at once)
      Cplx<float>* rf = (Cplx<float>*)r_s;
      const int co[4] = {c[0] - lc[0], c[1] - lc[1], c[2] - lc[2], c[3] - lc[3]};
      __syncthreads();
      smem_gather_dir<0>(rf, sg, g, delta, gauge, co, l, kappa);
      __syncthreads();
      smem_gather_dir<1>(rf, sg, g, delta, gauge, co, l, kappa);
      __syncthreads();
      smem_gather_dir<2>(rf, sg, g, delta, gauge, co, l, kappa);
      __syncthreads();
      smem_gather_dir<3>(rf, sg, g, delta, gauge, co, l, kappa);
      __syncthreads();
      r = rs_load<BF>(r_s, vb, l);
    }
  }

  Spinor<float> x;
#pragma unroll
  for (int k = 0; k < 12; k++) x.c[k] = cmk(0.f, 0.f);

  const int warp = l >> 5, lane = l & 31, nw = (vb + 31) >> 5;
  for (int step = 0; step < nmr; step++) {
    __syncthreads();
    Spinor<float> p = smem_clover_apply<S>(cl_s, vb, l, r);
    smem_block_hop<S, BF, 0>(p, r_s, lk_s, sg, l, lc, -kappa);
    smem_block_hop<S, BF, 1>(p, r_s, lk_s, sg, l, lc, -kappa);
    smem_block_hop<S, BF, 2>(p, r_s, lk_s, sg, l, lc, -kappa);
    smem_block_hop<S, BF, 3>(p, r_s, lk_s, sg, l, lc, -kappa);
    Cplx<float> pr = cmk(0.f, 0.f);
    float pp = 0;
#pragma unroll
    for (int k = 0; k < 12; k++) {
      cmac_conj(pr, p.c[k], r.c[k]);
      pp = fmaf(p.c[k].re, p.c[k].re, pp);
      pp = fmaf(p.c[k].im, p.c[k].im, pp);
    }
    float pr_re = pr.re, pr_im = pr.im;
    pr_re = warp_sum(pr_re);
    pr_im = warp_sum(pr_im);
    pp = warp_sum(pp);
    if (lane == 0) red[warp] = make_float4(pr_re, pr_im, pp, 0.f);
    __syncthreads();
    float a_re = 0, a_im = 0, n2 = 0;
    for (int w = 0; w < nw; w++) {
      const float4 v = red[w];
      a_re += v.x;
      a_im += v.y;
      n2 += v.z;
    }
    // a quotient, not a reciprocal: far from a point source both sums can be
    // denormal, where 1 / n2 overflows but a_re / n2 stays finite
    Cplx<float> alpha = n2 > 0.f ? cmk(a_re / n2, a_im / n2) : cmk(0.f, 0.f);
    const Cplx<float> malpha = -alpha;
#pragma unroll
    for (int k = 0; k < 12; k++) {
      cmac(x.c[k], alpha, r.c[k]);
      cmac(r.c[k], malpha, p.c[k]);
    }
    // every thread read its neighbours' residual for p before the barrier
    // above, so the new residual can be stored now; the next step's first
    // barrier orders the store (and the reads of red[]) before any later use
    rs_store<BF>(r_s, vb, l, r);
  }

  if (psi_init) {
    FieldsF::store_spinor(psi, g.V, s, x);
  } else {
    Spinor<float> y = FieldsF::load_spinor(psi, g.V, s);
#pragma unroll
    for (int k = 0; k < 12; k++) y.c[k] = y.c[k] + x.c[k];
    FieldsF::store_spinor(psi, g.V, s, y);
  }
  FieldsF::store_spinor(rho, g.V, s, r);
  FieldsF::store_spinor(delta, g.V, s, x);
}

template <typename F>
qcd_status launch_sweeps(qcd_ctx* c, const char* rho_src, char* rho, char* psi, char* delta, const void* gauge,
                         const void* clover, int nrhs, const int* mask, int nactive, int accumulate) {
  const qcd_solver_params& P = c->params;
  SapGeom sg;
  sg.vb = 1;
  for (int mu = 0; mu < 4; mu++) {
    sg.b[mu] = P.block[mu];
    sg.nb[mu] = c->g.L[mu] / sg.b[mu];
    sg.vb *= sg.b[mu];
  }
  sg.lst[1] = 1;
  sg.lst[2] = sg.b[1];
  sg.lst[3] = sg.b[1] * sg.b[2];
  sg.lst[0] = sg.b[1] * sg.b[2] * sg.b[3];
  const int nblocks = sg.nb[0] * sg.nb[1] * sg.nb[2] * sg.nb[3];
  const size_t smem = (size_t)12 * sg.vb * sizeof(Cplx<typename F::R>);
  // the register budget per thread follows from the block volume; FP32 fits
  // 128 registers without spilling, so 256-site blocks run two CTAs per SM
  constexpr int MINB256 = sizeof(typename F::R) == 4 ? 2 : 1;
  auto kern = sg.vb <= 256   ? k_sap_sweep<F, 256, MINB256>
              : sg.vb <= 512 ? k_sap_sweep<F, 512, 1>
                             : k_sap_sweep<F, 1024, 1>;
  QCD_CUDA_OK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const dim3 grid((unsigned)(nblocks / 2) * (unsigned)nrhs);
  // Algorithmic cost of one half-cycle (the minimum each launch must move):
  // per active site and RHS, rho read and written, psi read and written (only
  // written in the first cycle), delta written, and the other colour's delta
  // read once for every site that lies on a block face (fraction f_face of
  // the sites); per active site, once per launch, its 4 links and its clover
  // term.  Flops per active site and RHS: per MR step the block operator
  // (its internal hops and the clover term) plus the MR update (24 complex
  // multiply-adds), and one hop per face direction for the gather.
  double face = 0, inner = 1;
  for (int mu = 0; mu < 4; mu++) {
    face += 2.0 / sg.b[mu];
    inner *= 1.0 - 2.0 / sg.b[mu];
  }
  const double f_face = 1.0 - (inner > 0 ? inner : 0.0);
  const double sb = (double)F::spinor_bytes, lb = (double)F::link_bytes, cb = (double)F::clover_bytes;
  const double half = c->g.V / 2.0;
  const double flops_gather = 165.0 * face;
  const double flops_site = P.nmr * (1320.0 * (1.0 - face / 8.0) + 504.0 + 192.0) + flops_gather;
  const int fam = sizeof(typename F::R) == 8 ? FAM_SAP_D : FAM_SAP_F;
  // FP32 with blocks of at most 256 sites: the shared-memory-resident kernel
  const bool resident = sizeof(typename F::R) == 4 && sg.vb <= 256;
  const bool b4 = sg.b[0] == 4 && sg.b[1] == 4 && sg.b[2] == 4 && sg.b[3] == 4;
  auto kres = P.sap_half == 2   ? (b4 ? k_sap_sweep_smem<__half, true, true, 256, 2> : k_sap_sweep_smem<__half, true, false, 256, 2>)
              : P.sap_half == 1 ? (b4 ? k_sap_sweep_smem<__half, false, true, 256, 2>
                                      : k_sap_sweep_smem<__half, false, false, 256, 2>)
                                : (b4 ? k_sap_sweep_smem<float, false, true, 256, 1>
                                      : k_sap_sweep_smem<float, false, false, 256, 1>);
  const size_t smem_res = (size_t)sg.vb * ((P.sap_half == 2 ? 48 : 96) + (P.sap_half ? 144 + 144 : 288 + 288));
  // links and clover term read per active site and launch: their FP16 copies
  // (36 B per link, 144 B clover) for the 16-bit staged blocks, else FP32
  const double gcb = (resident && P.sap_half) ? 4 * 36.0 + 144.0 : 4 * lb + cb;
  if (resident)
    QCD_CUDA_OK(cudaFuncSetAttribute(kres, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_res));
  auto issue = [&]() -> qcd_status {
    for (int cy = 0; cy < P.ncy; cy++)
      for (int col = 0; col < 2; col++) {
        const int first = cy == 0 && !accumulate;
        const int gather = !(cy == 0 && col == 0);   // no boundary term before the first half-cycle
        const double bytes_rhs = sb * (2 + (first ? 1 : 2) + 1 + (gather ? f_face : 0.0));
        ProfScope ps(c, fam, half * (nactive * bytes_rhs + gcb),
                     half * nactive * (flops_site - (gather ? 0.0 : flops_gather)));
        const char* rin = cy == 0 ? rho_src : rho;   // the first cycle reads the caller's residual
        if (resident)
          kres<<<grid, sg.vb, smem_res, c->stream>>>(rin, rho, psi, delta, (const float4*)gauge, (const float4*)clover,
                                                     (const uint4*)c->gaugeH.p, (const uint4*)c->cloverH.p, c->g, sg,
                                                     col, gather, first, (float)c->kappa, P.nmr, nrhs, mask);
        else
          kern<<<grid, sg.vb, smem, c->stream>>>(rin, rho, psi, delta, gauge, clover, c->g, sg, col,
                                                 gather, first, (typename F::R)c->kappa, P.nmr, nrhs,
                                                 mask);
        QCD_CUDA_OK(cudaGetLastError());
      }
    return QCD_OK;
  };
  if (!P.graphs || c->stream == nullptr) return issue();
  // replay the whole application from a cached CUDA graph
  SapGraph key;
  key.rho_src = rho_src;
  key.rho = rho; key.psi = psi; key.delta = delta; key.gauge = gauge; key.clover = clover; key.mask = mask;
  key.nrhs = nrhs; key.ncy = P.ncy; key.nmr = P.nmr; key.accumulate = accumulate; key.half = P.sap_half;
  key.prec = (int)sizeof(typename F::R);
  for (int mu = 0; mu < 4; mu++) key.block[mu] = P.block[mu];
  key.kappa = c->kappa;
  cudaGraphExec_t exec = nullptr;
  for (auto& gph : c->sap_graphs)
    if (gph.rho_src == key.rho_src && gph.rho == key.rho && gph.psi == key.psi && gph.delta == key.delta && gph.gauge == key.gauge &&
        gph.clover == key.clover && gph.mask == key.mask && gph.nrhs == key.nrhs && gph.ncy == key.ncy &&
        gph.nmr == key.nmr && gph.accumulate == key.accumulate && gph.half == key.half && gph.prec == key.prec &&
        gph.kappa == key.kappa && memcmp(gph.block, key.block, sizeof(key.block)) == 0) {
      exec = gph.exec;
      break;
    }
  if (!exec) {
    cudaGraph_t graph = nullptr;
    QCD_CUDA_OK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    c->prof_suspend++;
    qcd_status st = issue();
    c->prof_suspend--;
    cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    if (st != QCD_OK) return st;
    QCD_CUDA_OK(e);
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    QCD_CUDA_OK(e);
    if (c->sap_graphs.size() >= 64) {
      cudaGraphExecDestroy(c->sap_graphs.front().exec);
      c->sap_graphs.erase(c->sap_graphs.begin());
    }
    key.exec = exec;
    c->sap_graphs.push_back(key);
  }
  double bytes = 0, flops = 0;
  for (int cy = 0; cy < P.ncy; cy++)
    for (int col = 0; col < 2; col++) {
      const int first = cy == 0 && !accumulate;
      const int gather = !(cy == 0 && col == 0);
      bytes += half * (nactive * sb * (2 + (first ? 1 : 2) + 1 + (gather ? f_face : 0.0)) + gcb);
      flops += half * nactive * (flops_site - (gather ? 0.0 : flops_gather));
    }
  ProfScope ps(c, fam, bytes, flops, 2 * P.ncy);
  QCD_CUDA_OK(cudaGraphLaunch(exec, c->stream));
  return QCD_OK;
}

}  // namespace

qcd_status sap_apply(qcd_ctx* c, void* rho, void* psi, void* delta, int prec, int nrhs, const int* mask,
                     int nactive, int accumulate, const void* rho_src) {
  const char* src = rho_src ? (const char*)rho_src : (const char*)rho;
  if (prec == QCD_PREC_F64)
    return launch_sweeps<FieldsD>(c, src, (char*)rho, (char*)psi, (char*)delta, c->gaugeD.p, c->cloverD.p, nrhs,
                                  mask, nactive, accumulate);
  return launch_sweeps<FieldsF>(c, src, (char*)rho, (char*)psi, (char*)delta, c->gaugeF.p, c->cloverF.p, nrhs, mask,
                                nactive, accumulate);
}
