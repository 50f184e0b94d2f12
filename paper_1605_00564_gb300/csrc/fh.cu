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
// P+- = (1 +- g0)/2 with g0_{i, i^2} = -1 in the chiral basis.  The two
// parities enter through one weighted projector per time-slice,
// Pw = conj(g+) P+ + conj(g-) P- = (1/2) [ws 1 - wd X], ws = conj(g+) + conj(g-),
// wd = conj(g+) - conj(g-), X_{i, i^2} = 1, whose derivative kernel
// (nucleon_grad.cuh) gives H_f = sum_{p,t} g(p,t) conj(dC(p,t)/dS_f).
#include <vector>

#include "nucleon_grad.cuh"

namespace {

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
  // weighted projector per timeslice: C_out[p][trel] = sign(t) c_p(t)
  std::vector<double2> pm(16 * (size_t)T);
  const int bc3 = c->g.bc_t * c->g.bc_t * c->g.bc_t;
  for (int t = 0; t < T; t++) {
    int trel = (t - src[0] + T) % T;
    double sg = t < src[0] ? (double)bc3 : 1.0;
    double2 gp = make_double2(sg * gcorr[2 * trel], sg * gcorr[2 * trel + 1]);
    double2 gm = make_double2(sg * gcorr[2 * (T + trel)], sg * gcorr[2 * (T + trel) + 1]);
    // ws = conj(g+) + conj(g-), wd = conj(g+) - conj(g-)
    const double2 ws = make_double2(gp.x + gm.x, -(gp.y + gm.y));
    const double2 wd = make_double2(gp.x - gm.x, -(gp.y - gm.y));
    for (int i = 0; i < 4; i++)
      for (int j = 0; j < 4; j++) {
        double2 v = make_double2(0.0, 0.0);
        if (i == j) v = make_double2(0.5 * ws.x, 0.5 * ws.y);
        if (j == (i ^ 2)) v = make_double2(v.x - 0.5 * wd.x, v.y - 0.5 * wd.y);
        pm[16 * (size_t)t + 4 * i + j] = v;
      }
  }
  QCD_TRY(devbuf_ensure(c->contract, sizeof(double2) * 16 * T));
  QCD_CUDA_OK(cudaMemcpyAsync(c->contract.p, pm.data(), sizeof(double2) * 16 * T, cudaMemcpyHostToDevice, c->stream));
  int ns = 8;
  while (L3 % ns) ns >>= 1;
  {
    ProfScope ps(c, FAM_CONTRACT, (double)V * (2304 + 2 * 2304), (double)V * 36 * 6 * 200 * 8);
    const size_t smem = sizeof(Cplx<double>) * 144 * ns;
    QCD_CUDA_OK(cudaFuncSetAttribute(nucleon_grad::k_dC_dS, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    nucleon_grad::k_dC_dS<<<V / ns, 18 * ns, smem, c->stream>>>((const double2*)c->wsD[4].p,
                                                               (const double2*)c->contract.p, V, L3, ns, 0,
                                                               (double2*)c->wsD[5].p);
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
  QCD_TRY(devbuf_ensure(c->small, sizeof(double2) * 48));
  double* dd = (double*)c->small.p;
  const char* Yu = (const char*)c->wsD[5].p;
  const char* Yd = Yu + f64 * 12;
  QCD_TRY(blas_dot(c, Yu, QCD_PREC_F64, c->wsD[4].p, QCD_PREC_F64, 12, dd, nullptr));
  QCD_TRY(blas_dot(c, Yd, QCD_PREC_F64, c->wsD[4].p, QCD_PREC_F64, 12, dd + 24, nullptr));
  QCD_TRY(blas_dot(c, Yu, QCD_PREC_F64, c->wsD[0].p, QCD_PREC_F64, 12, dd + 48, nullptr));
  QCD_TRY(blas_dot(c, Yd, QCD_PREC_F64, c->wsD[0].p, QCD_PREC_F64, 12, dd + 72, nullptr));
  std::vector<double> h(96);
  QCD_CUDA_OK(cudaMemcpyAsync(h.data(), dd, sizeof(double) * 96, cudaMemcpyDeviceToHost, c->stream));
  QCD_CUDA_OK(cudaStreamSynchronize(c->stream));
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
