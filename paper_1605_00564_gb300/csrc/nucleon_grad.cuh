// Derivative of the projected nucleon two-point contraction with respect to
// the point-source propagators of its quark lines, per site.  Shared by the
// Feynman-Hellmann gradient (fh.cu, weights over all time-slices) and the
// sequential sources of the three-point functions (threept.cu, one sink
// time-slice).
//
// C(x) = tr[P(t) G(x)] with G(x) = F(S_u, S_d, S_u)(x) the trilinear Wick
// form of eq. Nop (the diquark's u quark, the d quark, the third quark; the
// two Wick terms differ in which u-bar each u meets) and P(t) a 4x4 complex
// matrix per time-slice.  The kernel writes, for f = u and d,
//     H_f(x) = conj( dC(x) / dS_f(x) )          (12 x 12 per site)
// summed over the slots of flavour f, in the propagator's layout (field
// rhs = 3 alpha' + colour', component 3 alpha + colour).
//
// Gamma structure (chiral basis): G = C g5 = diag(J, J), J = [[0,-1],[1,0]],
// G' = g0 G^+ g0^T = -G; both act as "flip the index by ^1 and multiply by
// g(i) g(j)", g(b) = -1 for even b, +1 for odd b.
#pragma once

#include "qcd_internal.cuh"

namespace nucleon_grad {
namespace {

__constant__ int c_perm_fh[6][4] = {  // a, b, c, sign
    {0, 1, 2, 1}, {1, 2, 0, 1}, {2, 0, 1, 1}, {0, 2, 1, -1}, {2, 1, 0, -1}, {1, 0, 2, -1}};

using C64 = Cplx<double>;

__device__ inline double gs(int b) { return (b & 1) ? 1.0 : -1.0; }

struct M4 {
  C64 m[4][4];
};

__device__ inline M4 load_blk(const C64* S_s, int ns, int i, int x, int xp) {
  M4 o;
#pragma unroll
  for (int al = 0; al < 4; al++)
#pragma unroll
    for (int alp = 0; alp < 4; alp++) o.m[al][alp] = S_s[((3 * al + x) * 12 + 3 * alp + xp) * ns + i];
  return o;
}
__device__ inline M4 mm(const M4& a, const M4& b) {
  M4 o;
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) {
      C64 s = cmk(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < 4; k++) s = s + a.m[i][k] * b.m[k][j];
      o.m[i][j] = s;
    }
  return o;
}
// (G X G')-type sandwich: out_{ij} = g(i) g(j) X_{i^1, j^1}
__device__ inline M4 flip(const M4& X) {
  M4 o;
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) o.m[i][j] = (gs(i) * gs(j)) * X.m[i ^ 1][j ^ 1];
  return o;
}
// M = G'^T X^T G^T: M_{ij} = g(i) g(j) X_{j^1, i^1}
__device__ inline M4 flipT(const M4& X) {
  M4 o;
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) o.m[i][j] = (gs(i) * gs(j)) * X.m[j ^ 1][i ^ 1];
  return o;
}
__device__ inline C64 trace_prod(const M4& a, const M4& b) {   // tr[a b]
  C64 s = cmk(0.0, 0.0);
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int k = 0; k < 4; k++) s = s + a.m[i][k] * b.m[k][i];
  return s;
}

// H_f for NS sites per CTA, the CTAs covering the sites site0, site0 + 1, ...;
// thread = (site i, output o), o = 9 f + 3 x + x' holding the 4x4 spin block
// (x, x') of flavour f (0: u, 1: d).  pmat[t]: the 4x4 complex matrix P(t)
// (row major) of time-slice t.  prop: internal FP64 layout, 12 fields; H:
// internal FP64 layout, 24 fields (u then d), rhs = 3 alpha' + x'.
__global__ void k_dC_dS(const double2* __restrict__ prop, const double2* __restrict__ pmat, int V, int L3, int ns,
                        int site0, double2* __restrict__ H) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C64* S_s = (C64*)smem_raw;
  const int s0 = site0 + blockIdx.x * ns;
  for (int idx = threadIdx.x; idx < 144 * ns; idx += blockDim.x) {
    int i = idx % ns, e = idx / ns;
    int comp = e / 12, rhs = e - comp * 12;
    double2 v = prop[((size_t)rhs * 12 + comp) * V + s0 + i];
    S_s[e * ns + i] = cmk(v.x, v.y);
  }
  __syncthreads();
  const int i = threadIdx.x % ns, o = threadIdx.x / ns;
  if (o >= 18) return;
  const int f = o / 9, x = (o % 9) / 3, xp = o % 3;
  const int t = (s0 + i) / L3;
  M4 Pw;
#pragma unroll
  for (int u = 0; u < 4; u++)
#pragma unroll
    for (int v = 0; v < 4; v++) {
      const double2 e = pmat[16 * t + 4 * u + v];
      Pw.m[u][v] = cmk(e.x, e.y);
    }
  M4 acc;
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int b = 0; b < 4; b++) acc.m[a][b] = cmk(0.0, 0.0);
  for (int p = 0; p < 6; p++) {
    const int a = c_perm_fh[p][0], b = c_perm_fh[p][1], c = c_perm_fh[p][2];
    for (int q = 0; q < 6; q++) {
      const int ap = c_perm_fh[q][0], bp = c_perm_fh[q][1], cp = c_perm_fh[q][2];
      const double ee = (double)(c_perm_fh[p][3] * c_perm_fh[q][3]);
      // first Wick term: ee tr[Pw S^{cc'}] tr[S^{aa'T} G S^{bb'} G']
      if (f == 0 && x == a && xp == ap) {          // d/dS_u^{aa'} = ee trP(S^{cc'}) (G S^{bb'} G')
        C64 tp = trace_prod(Pw, load_blk(S_s, ns, i, c, cp));
        M4 Y = flip(load_blk(S_s, ns, i, b, bp));
        for (int u = 0; u < 4; u++)
          for (int v = 0; v < 4; v++) acc.m[u][v] = acc.m[u][v] + (ee * tp) * Y.m[u][v];
      }
      if (f == 0 && x == c && xp == cp) {          // d/dS_u^{cc'}_{al al'} = ee Pw_{al' al} T
        M4 A = load_blk(S_s, ns, i, a, ap), B = flip(load_blk(S_s, ns, i, b, bp));
        C64 T = cmk(0.0, 0.0);
        for (int u = 0; u < 4; u++)
          for (int v = 0; v < 4; v++) T = T + A.m[u][v] * B.m[u][v];
        for (int u = 0; u < 4; u++)
          for (int v = 0; v < 4; v++) acc.m[u][v] = acc.m[u][v] + (ee * T) * Pw.m[v][u];
      }
      if (f == 1 && x == b && xp == bp) {          // d/dS_d^{bb'} = ee trP(S^{cc'}) (G^T S^{aa'} G'^T)
        C64 tp = trace_prod(Pw, load_blk(S_s, ns, i, c, cp));
        M4 Y = flip(load_blk(S_s, ns, i, a, ap));
        for (int u = 0; u < 4; u++)
          for (int v = 0; v < 4; v++) acc.m[u][v] = acc.m[u][v] + (ee * tp) * Y.m[u][v];
      }
      // second Wick term (subtracted): ee tr[Pw S^{ca'} M S^{ac'}], M = G'^T S^{bb'T} G^T
      if (f == 0 && x == c && xp == ap) {          // d/dS_u^{ca'}_{jk} = ee (M S^{ac'} Pw)_{kj}
        M4 Z = mm(mm(flipT(load_blk(S_s, ns, i, b, bp)), load_blk(S_s, ns, i, a, cp)), Pw);
        for (int u = 0; u < 4; u++)
          for (int v = 0; v < 4; v++) acc.m[u][v] = acc.m[u][v] - ee * Z.m[v][u];
      }
      if (f == 0 && x == a && xp == cp) {          // d/dS_u^{ac'}_{jk} = ee (Pw S^{ca'} M)_{kj}
        M4 Z = mm(mm(Pw, load_blk(S_s, ns, i, c, ap)), flipT(load_blk(S_s, ns, i, b, bp)));
        for (int u = 0; u < 4; u++)
          for (int v = 0; v < 4; v++) acc.m[u][v] = acc.m[u][v] - ee * Z.m[v][u];
      }
      if (f == 1 && x == b && xp == bp) {          // d/dS_d^{bb'}_{nm} = ee (G^T (S^{ac'} Pw S^{ca'}) G'^T)_{nm}
        M4 Z = flip(mm(mm(load_blk(S_s, ns, i, a, cp), Pw), load_blk(S_s, ns, i, c, ap)));
        for (int u = 0; u < 4; u++)
          for (int v = 0; v < 4; v++) acc.m[u][v] = acc.m[u][v] - ee * Z.m[u][v];
      }
    }
  }
  // acc = dC/dS; H = conj(acc).  Entry (al, al') -> field rhs = 3 al' + x', comp 3 al + x
  double2* Hf = H + (size_t)f * 12 * 12 * V;
  for (int al = 0; al < 4; al++)
    for (int alp = 0; alp < 4; alp++)
      Hf[((size_t)(3 * alp + xp) * 12 + 3 * al + x) * V + s0 + i] = make_double2(acc.m[al][alp].re, -acc.m[al][alp].im);
}

}  // namespace
}  // namespace nucleon_grad

