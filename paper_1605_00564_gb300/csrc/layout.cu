// Field layouts: canonical FP64 <-> internal structure-of-arrays copies, and
// the clover term built from plaquette leaves on the device.
#include "qcd_internal.cuh"

namespace {

constexpr int TPB = 256;

inline int nblk(size_t n, int tpb = TPB) { return (int)((n + tpb - 1) / tpb); }

// canonical [site][mu][3][3] complex -> gaugeD double2[4][9][V], gaugeF float4[4][3][V]
__global__ void k_gauge_import(const double2* __restrict__ U, double2* __restrict__ gD, float4* __restrict__ gF,
                               int V) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
#pragma unroll
  for (int mu = 0; mu < 4; mu++) {
    double2 m[9];
#pragma unroll
    for (int k = 0; k < 9; k++) m[k] = U[((size_t)s * 4 + mu) * 9 + k];
#pragma unroll
    for (int k = 0; k < 9; k++) gD[((size_t)mu * 9 + k) * V + s] = m[k];
    float4* f = gF + (size_t)mu * 3 * V;
    f[s] = make_float4((float)m[0].x, (float)m[0].y, (float)m[1].x, (float)m[1].y);
    f[(size_t)V + s] = make_float4((float)m[2].x, (float)m[2].y, (float)m[3].x, (float)m[3].y);
    f[2 * (size_t)V + s] = make_float4((float)m[4].x, (float)m[4].y, (float)m[5].x, (float)m[5].y);
  }
}

using C64 = Cplx<double>;
using M3 = SU3<double>;

__device__ inline M3 mmul(const M3& a, const M3& b) {
  M3 o;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) o.m[i][j] = a.m[i][0] * b.m[0][j] + a.m[i][1] * b.m[1][j] + a.m[i][2] * b.m[2][j];
  return o;
}
__device__ inline M3 mdag(const M3& a) {
  M3 o;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) o.m[i][j] = conj(a.m[j][i]);
  return o;
}
__device__ inline M3 madd(const M3& a, const M3& b) {
  M3 o;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) o.m[i][j] = a.m[i][j] + b.m[i][j];
  return o;
}

// site index displaced by (dmu steps in mu, dnu steps in nu), steps in {-1,0,1}
__device__ inline int displaced(const Geom& g, const int c[4], int mu, int dmu, int nu, int dnu) {
  int cc[4] = {c[0], c[1], c[2], c[3]};
  cc[mu] = (cc[mu] + dmu + g.L[mu]) % g.L[mu];
  cc[nu] = (cc[nu] + dnu + g.L[nu]) % g.L[nu];
  return ((cc[0] * g.L[3] + cc[3]) * g.L[2] + cc[2]) * g.L[1] + cc[1];
}

__device__ inline M3 link(const double2* gD, int V, int mu, int s) {
  M3 U;
#pragma unroll
  for (int k = 0; k < 9; k++) {
    double2 v = gD[((size_t)mu * 9 + k) * V + s];
    U.m[k / 3][k % 3] = cmk(v.x, v.y);
  }
  return U;
}

// F_{mu nu}(x) = (Q - Q^+)/8, Q = the four leaves with a corner at x
__device__ M3 field_strength(const double2* gD, const Geom& g, int s, const int c[4], int mu, int nu) {
  int V = g.V;
  int xpm = displaced(g, c, mu, 1, nu, 0), xpn = displaced(g, c, mu, 0, nu, 1);
  int xmm = displaced(g, c, mu, -1, nu, 0), xmn = displaced(g, c, mu, 0, nu, -1);
  int xmm_pn = displaced(g, c, mu, -1, nu, 1), xpm_mn = displaced(g, c, mu, 1, nu, -1);
  int xmm_mn = displaced(g, c, mu, -1, nu, -1);
  M3 Um = link(gD, V, mu, s), Un = link(gD, V, nu, s);
  // leaf in the (+mu, +nu) quadrant
  M3 Q = mmul(mmul(Um, link(gD, V, nu, xpm)), mmul(mdag(link(gD, V, mu, xpn)), mdag(Un)));
  // (-mu, +nu)
  Q = madd(Q, mmul(mmul(Un, mdag(link(gD, V, mu, xmm_pn))), mmul(mdag(link(gD, V, nu, xmm)), link(gD, V, mu, xmm))));
  // (-mu, -nu)
  Q = madd(Q, mmul(mmul(mdag(link(gD, V, mu, xmm)), mdag(link(gD, V, nu, xmm_mn))),
                   mmul(link(gD, V, mu, xmm_mn), link(gD, V, nu, xmn))));
  // (+mu, -nu)
  Q = madd(Q, mmul(mmul(mdag(link(gD, V, nu, xmn)), link(gD, V, mu, xmn)), mmul(link(gD, V, nu, xpm_mn), mdag(Um))));
  M3 F;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) F.m[i][j] = 0.125 * (Q.m[i][j] - conj(Q.m[j][i]));
  return F;
}

// Pack a 6x6 Hermitian block [[1 + X3, X1 - i X2], [X1 + i X2, 1 - X3]]
// (X_l Hermitian 3x3) into 36 reals: diagonal, then lower triangle by rows.
__device__ void pack_block(const M3& X1, const M3& X2, const M3& X3, double* out) {
  C64 H[6][6];
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++) {
      C64 one = cmk(a == b ? 1.0 : 0.0, 0.0);
      H[a][b] = one + X3.m[a][b];
      H[3 + a][3 + b] = one - X3.m[a][b];
      H[a][3 + b] = X1.m[a][b] - mul_i(X2.m[a][b]);
      H[3 + a][b] = X1.m[a][b] + mul_i(X2.m[a][b]);
    }
#pragma unroll
  for (int i = 0; i < 6; i++) out[i] = H[i][i].re;
  int k = 6;
#pragma unroll
  for (int i = 1; i < 6; i++)
#pragma unroll
    for (int j = 0; j < i; j++) {
      out[k++] = H[i][j].re;
      out[k++] = H[i][j].im;
    }
}

// Clover term per site.  In the chiral basis sigma_{0k} = diag(s_k, -s_k) and
// sigma_{jk} = -eps_{jkl} diag(s_l, s_l), so
//   sum_{mu<nu} sigma F = diag( sum_l s_l B+_l , sum_l s_l B-_l )
//   B+ = (F01 - F23, F02 + F13, F03 - F12),  B- = (-F01 - F23, -F02 + F13, -F03 - F12)
// and the chiral blocks of A = 1 + i kappa c_sw sum sigma F are
//   1 + sum_l s_l X_l with X_l = i kappa c_sw B_l.
__global__ void k_clover_build(const double2* __restrict__ gD, Geom g, double kc, double2* __restrict__ clD,
                               float4* __restrict__ clF) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int c[4];
  site_coords(g, s, c);
  M3 F01 = field_strength(gD, g, s, c, 0, 1), F02 = field_strength(gD, g, s, c, 0, 2);
  M3 F03 = field_strength(gD, g, s, c, 0, 3), F12 = field_strength(gD, g, s, c, 1, 2);
  M3 F13 = field_strength(gD, g, s, c, 1, 3), F23 = field_strength(gD, g, s, c, 2, 3);
  double out[72];
  M3 X[3], Y[3];
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      C64 bp1 = F01.m[i][j] - F23.m[i][j], bp2 = F02.m[i][j] + F13.m[i][j], bp3 = F03.m[i][j] - F12.m[i][j];
      C64 bm1 = -F01.m[i][j] - F23.m[i][j], bm2 = -F02.m[i][j] + F13.m[i][j], bm3 = -F03.m[i][j] - F12.m[i][j];
      X[0].m[i][j] = kc * mul_i(bp1); X[1].m[i][j] = kc * mul_i(bp2); X[2].m[i][j] = kc * mul_i(bp3);
      Y[0].m[i][j] = kc * mul_i(bm1); Y[1].m[i][j] = kc * mul_i(bm2); Y[2].m[i][j] = kc * mul_i(bm3);
    }
  pack_block(X[0], X[1], X[2], out);
  pack_block(Y[0], Y[1], Y[2], out + 36);
#pragma unroll
  for (int k = 0; k < 36; k++) clD[(size_t)k * g.V + s] = make_double2(out[2 * k], out[2 * k + 1]);
#pragma unroll
  for (int k = 0; k < 18; k++)
    clF[(size_t)k * g.V + s] =
        make_float4((float)out[4 * k], (float)out[4 * k + 1], (float)out[4 * k + 2], (float)out[4 * k + 3]);
}

// packed blocks -> [site][2][6][6] complex
__global__ void k_clover_export(const double2* __restrict__ clD, int V, double2* __restrict__ out) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  double cl[72];
  for (int k = 0; k < 36; k++) {
    double2 v = clD[(size_t)k * V + s];
    cl[2 * k] = v.x;
    cl[2 * k + 1] = v.y;
  }
  for (int b = 0; b < 2; b++) {
    const double* p = cl + 36 * b;
    double2* o = out + ((size_t)s * 2 + b) * 36;
    for (int i = 0; i < 6; i++) o[i * 6 + i] = make_double2(p[i], 0.0);
    int k = 6;
    for (int i = 1; i < 6; i++)
      for (int j = 0; j < i; j++) {
        o[i * 6 + j] = make_double2(p[k], p[k + 1]);
        o[j * 6 + i] = make_double2(p[k], -p[k + 1]);
        k += 2;
      }
  }
}

// canonical [rhs][V][12] complex -> internal (prec 0: double2[rhs][12][V]; 1: float4[rhs][6][V])
template <typename T>
__global__ void k_spinor_import(const double2* __restrict__ in, T* __restrict__ out, int V, int nrhs);

template <>
__global__ void k_spinor_import<double2>(const double2* __restrict__ in, double2* __restrict__ out, int V, int nrhs) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)V * nrhs) return;
  int s = (int)(i % V);
  size_t r = i / V;
  const double2* p = in + i * 12;
#pragma unroll
  for (int c = 0; c < 12; c++) out[(r * 12 + c) * V + s] = p[c];
}
template <>
__global__ void k_spinor_import<float4>(const double2* __restrict__ in, float4* __restrict__ out, int V, int nrhs) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)V * nrhs) return;
  int s = (int)(i % V);
  size_t r = i / V;
  const double2* p = in + i * 12;
#pragma unroll
  for (int k = 0; k < 6; k++) {
    double2 a = p[2 * k], b = p[2 * k + 1];
    out[(r * 6 + k) * V + s] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
  }
}

template <typename T>
__global__ void k_spinor_export(const T* __restrict__ in, double2* __restrict__ out, int V, int nrhs);

template <>
__global__ void k_spinor_export<double2>(const double2* __restrict__ in, double2* __restrict__ out, int V, int nrhs) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)V * nrhs) return;
  int s = (int)(i % V);
  size_t r = i / V;
  double2* p = out + i * 12;
#pragma unroll
  for (int c = 0; c < 12; c++) p[c] = in[(r * 12 + c) * V + s];
}
template <>
__global__ void k_spinor_export<float4>(const float4* __restrict__ in, double2* __restrict__ out, int V, int nrhs) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)V * nrhs) return;
  int s = (int)(i % V);
  size_t r = i / V;
  double2* p = out + i * 12;
#pragma unroll
  for (int k = 0; k < 6; k++) {
    float4 v = in[(r * 6 + k) * V + s];
    p[2 * k] = make_double2(v.x, v.y);
    p[2 * k + 1] = make_double2(v.z, v.w);
  }
}

// FP16 copies of the FP32 links (full 3x3) and clover term, rounded exactly as
// the SAP kernel's staging rounds them (one conversion per (re, im) pair)
__global__ void k_half_fields(const float4* __restrict__ gaugeF, const float4* __restrict__ cloverF, int V,
                              uint4* __restrict__ gA, uint4* __restrict__ gB, unsigned* __restrict__ gC,
                              uint4* __restrict__ clH) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  for (int mu = 0; mu < 4; mu++) {
    const SU3<float> U = FieldsF::load_link(gaugeF, V, mu, s);
    unsigned h[9];
    for (int k = 0; k < 9; k++) h[k] = h2_bits(__floats2half2_rn(U.m[k / 3][k % 3].re, U.m[k / 3][k % 3].im));
    gA[(size_t)mu * V + s] = make_uint4(h[0], h[1], h[2], h[3]);
    gB[(size_t)mu * V + s] = make_uint4(h[4], h[5], h[6], h[7]);
    gC[(size_t)mu * V + s] = h[8];
  }
  for (int k = 0; k < 9; k++) {
    const float4 a = cloverF[(size_t)(2 * k) * V + s], b = cloverF[(size_t)(2 * k + 1) * V + s];
    clH[(size_t)k * V + s] = make_uint4(h2_bits(__floats2half2_rn(a.x, a.y)), h2_bits(__floats2half2_rn(a.z, a.w)),
                                        h2_bits(__floats2half2_rn(b.x, b.y)), h2_bits(__floats2half2_rn(b.z, b.w)));
  }
}

}  // namespace

qcd_status layout_gauge_import(qcd_ctx* c, const double* U_dev) {
  int V = c->g.V;
  QCD_TRY(devbuf_ensure(c->gaugeD, (size_t)V * 4 * 9 * sizeof(double2)));
  QCD_TRY(devbuf_ensure(c->gaugeF, (size_t)V * 4 * 3 * sizeof(float4)));
  ProfScope ps(c, FAM_LAYOUT, (double)V * (576 + 576 + 192), 0.0);
  k_gauge_import<<<nblk(V), TPB, 0, c->stream>>>((const double2*)U_dev, (double2*)c->gaugeD.p, (float4*)c->gaugeF.p,
                                                 V);
  QCD_CUDA_OK(cudaGetLastError());
  return QCD_OK;
}

qcd_status layout_clover_build(qcd_ctx* c) {
  int V = c->g.V;
  QCD_TRY(devbuf_ensure(c->cloverD, (size_t)V * 36 * sizeof(double2)));
  QCD_TRY(devbuf_ensure(c->cloverF, (size_t)V * 18 * sizeof(float4)));
  ProfScope ps(c, FAM_LAYOUT, (double)V * (576 + 576 + 288), 0.0);
  k_clover_build<<<nblk(V, 128), 128, 0, c->stream>>>((const double2*)c->gaugeD.p, c->g, c->kappa * c->csw,
                                                      (double2*)c->cloverD.p, (float4*)c->cloverF.p);
  QCD_CUDA_OK(cudaGetLastError());
  // FP16 copies of links and clover term for the sloppy SAP block solves
  QCD_TRY(devbuf_ensure(c->gaugeH, (size_t)V * 4 * 36));
  QCD_TRY(devbuf_ensure(c->cloverH, (size_t)V * 144));
  uint4* gA = (uint4*)c->gaugeH.p;
  uint4* gB = gA + 4 * (size_t)V;
  unsigned* gC = (unsigned*)(gB + 4 * (size_t)V);
  k_half_fields<<<nblk(V, 128), 128, 0, c->stream>>>((const float4*)c->gaugeF.p, (const float4*)c->cloverF.p, V, gA,
                                                     gB, gC, (uint4*)c->cloverH.p);
  QCD_CUDA_OK(cudaGetLastError());
  return QCD_OK;
}

qcd_status clover_export(qcd_ctx* c, double* out_dev) {
  k_clover_export<<<nblk(c->g.V, 128), 128, 0, c->stream>>>((const double2*)c->cloverD.p, c->g.V, (double2*)out_dev);
  QCD_CUDA_OK(cudaGetLastError());
  return QCD_OK;
}

qcd_status layout_spinor_import(qcd_ctx* c, const double* in, void* out, int prec, int nrhs) {
  size_t n = (size_t)c->g.V * nrhs;
  ProfScope ps(c, FAM_LAYOUT, (double)n * (192 + (prec == QCD_PREC_F64 ? 192 : 96)), 0.0);
  if (prec == QCD_PREC_F64)
    k_spinor_import<double2><<<nblk(n), TPB, 0, c->stream>>>((const double2*)in, (double2*)out, c->g.V, nrhs);
  else
    k_spinor_import<float4><<<nblk(n), TPB, 0, c->stream>>>((const double2*)in, (float4*)out, c->g.V, nrhs);
  QCD_CUDA_OK(cudaGetLastError());
  return QCD_OK;
}

qcd_status layout_spinor_export(qcd_ctx* c, const void* in, double* out, int prec, int nrhs) {
  size_t n = (size_t)c->g.V * nrhs;
  ProfScope ps(c, FAM_LAYOUT, (double)n * (192 + (prec == QCD_PREC_F64 ? 192 : 96)), 0.0);
  if (prec == QCD_PREC_F64)
    k_spinor_export<double2><<<nblk(n), TPB, 0, c->stream>>>((const double2*)in, (double2*)out, c->g.V, nrhs);
  else
    k_spinor_export<float4><<<nblk(n), TPB, 0, c->stream>>>((const float4*)in, (double2*)out, c->g.V, nrhs);
  QCD_CUDA_OK(cudaGetLastError());
  return QCD_OK;
}

size_t spinor_bytes(const qcd_ctx* c, int prec) {
  return (size_t)c->g.V * (prec == QCD_PREC_F64 ? 192 : prec == QCD_PREC_H16 ? FieldsH::spinor_bytes : 96);
}
