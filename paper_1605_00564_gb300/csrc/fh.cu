// Derivatives of the nucleon two-point function with respect to the bare
// quark mass m0 and an isovector axial Feynman-Hellmann coupling lambda
// (D_w -> D_w + lambda g3 g5 for u, - lambda g3 g5 for d; the zero-momentum
// A_3 insertion of R_A, Sec. 2.3), by the adjoint method:
//
//   C(t) = F(S_u, S_d, S_u) is trilinear in the point-source propagators (the
//   diquark u quark, the d quark, the third quark).  For a real loss L with
//   upstream gradient g(p,t) = dL/dRe C + i dL/dIm C,
//     H_f(x) = sum_{p,t} g(p,t) conj(dC(p,t)/dS_f(x))      (this file's kernel)
//     Y_f    = (D_w^+)^-1 H_f = 2 kappa g5 D^-1 g5 H_f    (gamma_5-hermiticity)
//     dL/dtheta = -Re sum_x tr[Y_f(x)^+ (dD_w/dtheta)(x) S(x)]  summed over f,
//   with dD_w/dm0 = 1 and dD_w/dlambda = +g3 g5 (u), -g3 g5 (d).  Wilson
//   normalisation: S = D_w^-1 = 2 kappa D^-1 with D the kappa-normalised
//   operator of the library.
//
// Gamma structure (chiral basis): G = C g5 = diag(J, J), J = [[0,-1],[1,0]],
// G' = g0 G^+ g0^T = -G; both act as "flip the index by ^1 and multiply by
// g(i) g(j)", g(b) = -1 for even b, +1 for odd b.  P+- = (1 +- g0)/2 with
// g0_{i, i^2} = -1.  The two parities enter through one weighted projector
// Pw = conj(g+) P+ + conj(g-) P- = (1/2) [ws 1 - wd X], ws = conj(g+) + conj(g-),
// wd = conj(g+) - conj(g-), X_{i, i^2} = 1.
#include <vector>

#include "qcd_internal.cuh"

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
// Pw as a matrix
__device__ inline M4 pw_matrix(C64 ws, C64 wd) {
  M4 o;
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) {
      C64 v = cmk(0.0, 0.0);
      if (i == j) v = 0.5 * ws;
      if (j == (i ^ 2)) v = v - 0.5 * wd;
      o.m[i][j] = v;
    }
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

// H_f for NS sites per CTA; thread = (site i, output o), o = 9 f + 3 x + x'
// holding the 4x4 spin block (x, x') of flavour f (0: u, 1: d).
// gw[t] = (ws, wd) for timeslice t.  prop: internal FP64 layout, 12 fields;
// H: internal FP64 layout, 24 fields (u then d), rhs = 3 alpha' + x'.
__global__ void k_nucleon_bwd(const double2* __restrict__ prop, const double2* __restrict__ gw, int V, int L3, int ns,
                              double2* __restrict__ H) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C64* S_s = (C64*)smem_raw;
  const int s0 = blockIdx.x * ns;
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
  const double2 w0 = gw[2 * t], w1 = gw[2 * t + 1];
  const M4 Pw = pw_matrix(cmk(w0.x, w0.y), cmk(w1.x, w1.y));
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
  // acc = sum_p conj(g_p) dC_p/dS; H = conj(acc).  Entry (al, al') -> field rhs = 3 al' + x', comp 3 al + x
  double2* Hf = H + (size_t)f * 12 * 12 * V;
  for (int al = 0; al < 4; al++)
    for (int alp = 0; alp < 4; alp++)
      Hf[((size_t)(3 * alp + xp) * 12 + 3 * al + x) * V + s0 + i] = make_double2(acc.m[al][alp].re, -acc.m[al][alp].im);
}

// out = scale G in for G = g5 (which 0), g3 g5 (which 1) or 1 (which 2), internal FP64 layout
__global__ void k_gamma(const double2* __restrict__ in, double2* __restrict__ out, int which, double scale, int V,
                        int nrhs) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)V * nrhs) return;
  const size_t r = idx / V, s = idx % V;
  const double2* p = in + r * 12 * V + s;
  double2* q = out + r * 12 * V + s;
  for (int a = 0; a < 3; a++) {
    double2 v0 = p[(size_t)(0 + a) * V], v1 = p[(size_t)(3 + a) * V], v2 = p[(size_t)(6 + a) * V],
            v3 = p[(size_t)(9 + a) * V];
    double2 o0, o1, o2, o3;
    if (which == 2) {            // identity (scaling only)
      o0 = v0; o1 = v1; o2 = v2; o3 = v3;
    } else if (which == 0) {     // g5 = diag(1, 1, -1, -1)
      o0 = v0; o1 = v1;
      o2 = make_double2(-v2.x, -v2.y); o3 = make_double2(-v3.x, -v3.y);
    } else {                     // g3 g5 = [[0, i s3], [i s3, 0]], i s3 = diag(i, -i)
      o0 = make_double2(-v2.y, v2.x);   // i psi_2
      o1 = make_double2(v3.y, -v3.x);   // -i psi_3
      o2 = make_double2(-v0.y, v0.x);   // i psi_0
      o3 = make_double2(v1.y, -v1.x);   // -i psi_1
    }
    q[(size_t)(0 + a) * V] = make_double2(scale * o0.x, scale * o0.y);
    q[(size_t)(3 + a) * V] = make_double2(scale * o1.x, scale * o1.y);
    q[(size_t)(6 + a) * V] = make_double2(scale * o2.x, scale * o2.y);
    q[(size_t)(9 + a) * V] = make_double2(scale * o3.x, scale * o3.y);
  }
}

qcd_status gamma_apply(qcd_ctx* c, const void* in, void* out, int which, double scale, int nrhs) {
  size_t n = (size_t)c->g.V * nrhs;
  ProfScope ps(c, FAM_LAYOUT, (double)n * 2 * 192, 0.0);
  k_gamma<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>((const double2*)in, (double2*)out, which, scale,
                                                              c->g.V, nrhs);
  QCD_CUDA_OK(cudaGetLastError());
  return QCD_OK;
}

}  // namespace

qcd_status solver_run(qcd_ctx* c, int n, const double* tol, qcd_rhs_stats* st);
qcd_status contract_nucleon(qcd_ctx* c, const void* prop, int t0, double* corr_dev, int precision,
                            double2* partials);

namespace {
__global__ void k_point12(double2* eta, int V, int site) {
  int r = threadIdx.x;
  if (r < 12) eta[((size_t)r * 12 + r) * V + site] = make_double2(1.0, 0.0);
}
}  // namespace

extern "C" qcd_status qcd_fh_forward(qcd_ctx* c, const int src[4], double tol, double* prop, double* corr,
                                     qcd_rhs_stats* stats) {
  if (!c || !src || !prop || !corr || !(tol > 0 && tol < 1)) {
    qcd_set_error("bad argument");
    return QCD_ERR_ARG;
  }
  if (!c->have_gauge) {
    qcd_set_error("no gauge field loaded");
    return QCD_ERR_STATE;
  }
  for (int mu = 0; mu < 4; mu++)
    if (src[mu] < 0 || src[mu] >= c->g.L[mu]) {
      qcd_set_error("source outside the lattice");
      return QCD_ERR_ARG;
    }
  const size_t f64 = spinor_bytes(c, QCD_PREC_F64);
  const int T = c->g.L[0];
  QCD_TRY(devbuf_ensure(c->wsD[0], f64 * 12));
  QCD_TRY(devbuf_ensure(c->wsD[1], f64 * 12));
  QCD_TRY(devbuf_ensure(c->wsD[4], f64 * 12));
  QCD_CUDA_OK(cudaMemsetAsync(c->wsD[0].p, 0, f64 * 12, c->stream));
  QCD_CUDA_OK(cudaMemsetAsync(c->wsD[1].p, 0, f64 * 12, c->stream));
  const int site = ((src[0] * c->g.L[3] + src[3]) * c->g.L[2] + src[2]) * c->g.L[1] + src[1];
  k_point12<<<1, 32, 0, c->stream>>>((double2*)c->wsD[0].p, c->g.V, site);
  QCD_CUDA_OK(cudaGetLastError());
  std::vector<double> tols(12, tol);
  std::vector<qcd_rhs_stats> st(12);
  QCD_TRY(solver_run(c, 12, tols.data(), st.data()));
  // Wilson normalisation S = D_w^-1 = 2 kappa D^-1
  QCD_TRY(gamma_apply(c, c->wsD[1].p, c->wsD[4].p, 2, 2.0 * c->kappa, 12));
  QCD_TRY(layout_spinor_export(c, c->wsD[4].p, prop, QCD_PREC_F64, 12));
  const size_t npart = 2 * (size_t)c->g.V;
  QCD_TRY(devbuf_ensure(c->contract, sizeof(double2) * (npart + 2 * T)));
  double2* part = (double2*)c->contract.p;
  QCD_TRY(contract_nucleon(c, c->wsD[4].p, src[0], (double*)(part + npart), QCD_PREC_F64, part));
  QCD_CUDA_OK(cudaMemcpyAsync(corr, part + npart, sizeof(double2) * 2 * T, cudaMemcpyDeviceToHost, c->stream));
  QCD_CUDA_OK(cudaStreamSynchronize(c->stream));
  qcd_status worst = QCD_OK;
  for (int r = 0; r < 12; r++) {
    if (stats) stats[r] = st[r];
    if (st[r].status != QCD_OK && worst == QCD_OK) worst = (qcd_status)st[r].status;
  }
  return worst;
}

extern "C" qcd_status qcd_fh_gradient(qcd_ctx* c, const double* prop, const int src[4], const double* gcorr,
                                      double tol, double* grad, qcd_rhs_stats* stats) {
  if (!c || !prop || !src || !gcorr || !grad || !(tol > 0 && tol < 1)) {
    qcd_set_error("bad argument");
    return QCD_ERR_ARG;
  }
  if (!c->have_gauge) {
    qcd_set_error("no gauge field loaded");
    return QCD_ERR_STATE;
  }
  for (int mu = 0; mu < 4; mu++)
    if (src[mu] < 0 || src[mu] >= c->g.L[mu]) {
      qcd_set_error("source outside the lattice");
      return QCD_ERR_ARG;
    }
  const int V = c->g.V, T = c->g.L[0], L3 = V / T;
  const size_t f64 = spinor_bytes(c, QCD_PREC_F64);
  // workspaces: S (12), H (24) -> eta of the adjoint solve, X (24) = psi, G3G5 S (12)
  QCD_TRY(devbuf_ensure(c->wsD[4], f64 * 12));
  QCD_TRY(devbuf_ensure(c->wsD[5], f64 * 24));
  QCD_TRY(devbuf_ensure(c->wsD[0], f64 * 24));
  QCD_TRY(devbuf_ensure(c->wsD[1], f64 * 24));
  QCD_TRY(layout_spinor_import(c, prop, c->wsD[4].p, QCD_PREC_F64, 12));
  // weights per timeslice: C_out[p][trel] = sign(t) c_p(t)
  std::vector<double2> gw(2 * T);
  const int bc3 = c->g.bc_t * c->g.bc_t * c->g.bc_t;
  for (int t = 0; t < T; t++) {
    int trel = (t - src[0] + T) % T;
    double sg = t < src[0] ? (double)bc3 : 1.0;
    double2 gp = make_double2(sg * gcorr[2 * trel], sg * gcorr[2 * trel + 1]);
    double2 gm = make_double2(sg * gcorr[2 * (T + trel)], sg * gcorr[2 * (T + trel) + 1]);
    // conj(g+) + conj(g-), conj(g+) - conj(g-)
    gw[2 * t] = make_double2(gp.x + gm.x, -(gp.y + gm.y));
    gw[2 * t + 1] = make_double2(gp.x - gm.x, -(gp.y - gm.y));
  }
  QCD_TRY(devbuf_ensure(c->contract, sizeof(double2) * 2 * T));
  QCD_CUDA_OK(cudaMemcpyAsync(c->contract.p, gw.data(), sizeof(double2) * 2 * T, cudaMemcpyHostToDevice, c->stream));
  int ns = 8;
  while (L3 % ns) ns >>= 1;
  {
    ProfScope ps(c, FAM_CONTRACT, (double)V * (2304 + 2 * 2304), (double)V * 36 * 6 * 200 * 8);
    const size_t smem = sizeof(C64) * 144 * ns;
    QCD_CUDA_OK(cudaFuncSetAttribute(k_nucleon_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_nucleon_bwd<<<V / ns, 18 * ns, smem, c->stream>>>((const double2*)c->wsD[4].p, (const double2*)c->contract.p,
                                                       V, L3, ns, (double2*)c->wsD[5].p);
    QCD_CUDA_OK(cudaGetLastError());
  }
  // adjoint solve: X = D^-1 g5 H, Y = 2 kappa g5 X
  QCD_TRY(gamma_apply(c, c->wsD[5].p, c->wsD[0].p, 0, 1.0, 24));
  QCD_CUDA_OK(cudaMemsetAsync(c->wsD[1].p, 0, f64 * 24, c->stream));
  std::vector<double> tols(24, tol);
  std::vector<qcd_rhs_stats> st(24);
  QCD_TRY(solver_run(c, 24, tols.data(), st.data()));
  const double k2 = 2.0 * c->kappa;
  QCD_TRY(gamma_apply(c, c->wsD[1].p, c->wsD[5].p, 0, k2, 24));      // Y (u then d) into wsD[5]
  // S in Wilson normalisation is the input prop; (g3 g5) S into wsD[0]
  QCD_TRY(gamma_apply(c, c->wsD[4].p, c->wsD[0].p, 1, 1.0, 12));
  // dots per column: <Y_u, S>, <Y_d, S>, <Y_u, G S>, <Y_d, G S>
  double* dd = nullptr;
  QCD_CUDA_OK(cudaMallocAsync((void**)&dd, sizeof(double2) * 48, c->stream));
  const char* Yu = (const char*)c->wsD[5].p;
  const char* Yd = Yu + f64 * 12;
  QCD_TRY(blas_dot(c, Yu, QCD_PREC_F64, c->wsD[4].p, QCD_PREC_F64, 12, dd, nullptr));
  QCD_TRY(blas_dot(c, Yd, QCD_PREC_F64, c->wsD[4].p, QCD_PREC_F64, 12, dd + 24, nullptr));
  QCD_TRY(blas_dot(c, Yu, QCD_PREC_F64, c->wsD[0].p, QCD_PREC_F64, 12, dd + 48, nullptr));
  QCD_TRY(blas_dot(c, Yd, QCD_PREC_F64, c->wsD[0].p, QCD_PREC_F64, 12, dd + 72, nullptr));
  std::vector<double> h(96);
  QCD_CUDA_OK(cudaMemcpyAsync(h.data(), dd, sizeof(double) * 96, cudaMemcpyDeviceToHost, c->stream));
  QCD_CUDA_OK(cudaStreamSynchronize(c->stream));
  QCD_CUDA_OK(cudaFreeAsync(dd, c->stream));
  double dm = 0, dl = 0;
  for (int r = 0; r < 12; r++) {
    dm -= h[2 * r] + h[24 + 2 * r];          // -Re <Y_u + Y_d, S>
    dl += -h[48 + 2 * r] + h[72 + 2 * r];    // -Re <Y_u, G S> + Re <Y_d, G S>
  }
  grad[0] = dm;
  grad[1] = dl;
  qcd_status worst = QCD_OK;
  for (int r = 0; r < 24; r++) {
    if (stats) stats[r] = st[r];
    if (st[r].status != QCD_OK && worst == QCD_OK) worst = (qcd_status)st[r].status;
  }
  return worst;
}
