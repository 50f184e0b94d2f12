// Flexible GCR with the SAP preconditioner (Sec. 2.2): solve D M_SAP phi = eta,
// psi = M_SAP phi, for a batch of right-hand sides at once.
//
// Mixed precision (Sec. 2.2, last paragraph: the SAP preconditioner in single
// precision, parts of GCR in single precision): psi, rho and eta are FP64;
// the preconditioner, the Krylov vectors phi_k and chi_k = D phi_k are in
// the "inner" precision (FP32, or FP64 for the plain double-precision path).
// A restart cycle ends when the recursive residual has fallen by
// restart_drop (or after nkv vectors); then psi is updated and the residual
// is recomputed from its definition rho = eta - D psi with the FP64 operator.
//
// Within a cycle, chi_k = D phi_k is orthonormalised against chi_0..chi_{k-1}
// (classical Gram-Schmidt, coefficients a_kj), b_k = |chi_k|, c_k = (chi_k, rho),
// rho -= c_k chi_k.  Since D phi_k = b_k chi_k + sum_{j<k} a_kj chi_j, the
// coefficients alpha of psi += sum alpha_j phi_j solve the triangular system
// alpha_j b_j + sum_{k>j} alpha_k a_kj = c_j (back substitution on the host).
//
// Per right-hand side convergence: a device mask freezes the RHS that left
// the cycle (converged or dropped by restart_drop); all kernels skip masked
// RHS.  The only host reads are the residual norms once per iteration and the
// small coefficient arrays once per cycle.
#include <math.h>
#include <string.h>

#include <vector>

#include "qcd_internal.cuh"

namespace {

// b = |chi_k|, inv = 1/b, c_k = (chi_k, rho) / b from n2c = {|chi_k|^2, (chi_k, rho)}
__global__ void k_gs_scalars(const double2* n2c, double* b, double* inv, double2* ck, int n, const int* mask) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n || (mask && !mask[r])) return;
  double v = sqrt(n2c[r].x);
  double iv = v > 0 ? 1.0 / v : 0.0;
  b[r] = v;
  inv[r] = iv;
  ck[r] = make_double2(n2c[n + r].x * iv, n2c[n + r].y * iv);
}

struct Work {
  char *eta, *psi, *rho, *tmp;      // FP64 internal [n]
  char *rhoS, *delta, *sapin;       // inner precision [n]: recursive residual, SAP scratch
  char *phi, *chi;                  // inner precision [nkv][n]
  double2 *a;                       // [nkv][nkv][n]: a[k][j][r]
  double *b, *inv, *rn2;            // [nkv][n], [n], [n]
  double2 *n2c, *rn2c;              // [2][n], [n]
  double2 *cc, *alpha;              // [nkv][n]
  int* mask;                        // [n]
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

qcd_status get_work(qcd_ctx* c, int n, int nkv, int prec, int pchi, Work& w) {
  const size_t VD = spinor_bytes(c, QCD_PREC_F64) * n;
  const size_t VI = spinor_bytes(c, prec) * n;
  const size_t VC = align256(spinor_bytes(c, pchi) * n);
  DevBuf* bufD = c->wsD;
  QCD_TRY(devbuf_ensure(bufD[0], VD));
  QCD_TRY(devbuf_ensure(bufD[1], VD));
  QCD_TRY(devbuf_ensure(bufD[2], VD));
  QCD_TRY(devbuf_ensure(bufD[3], VD));
  w.eta = (char*)bufD[0].p;
  w.psi = (char*)bufD[1].p;
  w.rho = (char*)bufD[2].p;
  w.tmp = (char*)bufD[3].p;
  DevBuf& basis = prec == QCD_PREC_F64 ? c->basisD : c->basisF;
  QCD_TRY(devbuf_ensure(basis, VI * (nkv + 3) + VC * nkv));
  w.rhoS = (char*)basis.p;
  w.delta = w.rhoS + VI;
  w.sapin = w.delta + VI;
  w.phi = w.sapin + VI;
  w.chi = w.phi + VI * nkv;        // nkv vectors of VC bytes (chi's own storage)
  size_t sz = align256(sizeof(double2) * nkv * nkv * n) + align256(sizeof(double) * nkv * n) +
              2 * align256(sizeof(double) * n) + 2 * align256(sizeof(double2) * nkv * n) +
              align256(sizeof(double2) * 3 * n) + align256(sizeof(int) * n);
  QCD_TRY(devbuf_ensure(c->scal, sz));
  char* p = (char*)c->scal.p;
  w.a = (double2*)p;  p += align256(sizeof(double2) * nkv * nkv * n);
  w.b = (double*)p;   p += align256(sizeof(double) * nkv * n);
  w.inv = (double*)p; p += align256(sizeof(double) * n);
  w.rn2 = (double*)p; p += align256(sizeof(double) * n);
  w.n2c = (double2*)p; w.rn2c = w.n2c + 2 * n; p += align256(sizeof(double2) * 3 * n);
  w.cc = (double2*)p; p += align256(sizeof(double2) * nkv * n);
  w.alpha = (double2*)p; p += align256(sizeof(double2) * nkv * n);
  w.mask = (int*)p;
  return QCD_OK;
}

qcd_status host_mirror(qcd_ctx* c, size_t bytes) {
  if (c->host_scal_bytes >= bytes) return QCD_OK;
  if (c->host_scal) cudaFreeHost(c->host_scal);
  c->host_scal = nullptr;
  c->host_scal_bytes = 0;
  QCD_CUDA_OK(cudaMallocHost((void**)&c->host_scal, bytes));
  c->host_scal_bytes = bytes;
  return QCD_OK;
}

qcd_status fetch(qcd_ctx* c, void* host, const void* dev, size_t bytes) {
  QCD_CUDA_OK(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, c->stream));
  QCD_CUDA_OK(cudaStreamSynchronize(c->stream));
  return QCD_OK;
}

}  // namespace

// Solve for n right-hand sides already in the internal FP64 layout in the
// context workspace (eta -> wsD[0], initial guess -> wsD[1]); the solution is
// left in wsD[1].
qcd_status solver_run(qcd_ctx* c, int n, const double* tol, qcd_rhs_stats* st) {
  const qcd_solver_params& P = c->params;
  const int nkv = P.nkv, prec = P.precision;
  const bool use_dfl = P.dfl && dfl_ready(c) && prec == QCD_PREC_F32;
  // storage of the Krylov images chi_k: FP16 + per-site scale with basis_half
  const int pchi = (prec == QCD_PREC_F32 && P.basis_half) ? QCD_PREC_H16 : prec;
  Work w;
  QCD_TRY(get_work(c, n, nkv, prec, pchi, w));
  const size_t VI = spinor_bytes(c, prec) * n;
  const size_t VC = align256(spinor_bytes(c, pchi) * n);
  QCD_TRY(host_mirror(c, sizeof(double) * (8 * n + nkv * nkv * n * 2 + 4 * nkv * n * 2) + 64));
  double* h_rn2 = c->host_scal;
  double* h_eta = h_rn2 + n;
  double2* h_rn2c = (double2*)(h_eta + n);
  double2* h_a = h_rn2c + n;
  double* h_b = (double*)(h_a + (size_t)nkv * nkv * n);
  double2* h_c = (double2*)(h_b + (size_t)nkv * n);
  double2* h_alpha = h_c + (size_t)nkv * n;
  int* h_mask = (int*)(h_alpha + (size_t)nkv * n);

  std::vector<int> active(n, 1), incyc(n, 0), kcount(n, 0);
  std::vector<double> etan(n), r0(n);
  for (int r = 0; r < n; r++) {
    st[r].status = QCD_OK;
    st[r].outer_iters = 0;
    st[r].restarts = 0;
    st[r].true_rel_residual = 0;
  }

  QCD_TRY(blas_norm2(c, w.eta, QCD_PREC_F64, n, w.rn2, nullptr));
  QCD_TRY(fetch(c, h_eta, w.rn2, sizeof(double) * n));
  for (int r = 0; r < n; r++) {
    etan[r] = sqrt(h_eta[r]);
    if (!isfinite(etan[r])) {
      st[r].status = QCD_ERR_NONFINITE;
      active[r] = 0;
    } else if (etan[r] == 0.0) {
      active[r] = 0;   // psi = 0 is the exact solution
    }
  }
  auto upload_mask = [&](const std::vector<int>& m) -> qcd_status {
    for (int r = 0; r < n; r++) h_mask[r] = m[r];
    QCD_CUDA_OK(cudaMemcpyAsync(w.mask, h_mask, sizeof(int) * n, cudaMemcpyHostToDevice, c->stream));
    return QCD_OK;
  };
  // zero-norm sources: psi = 0
  {
    std::vector<int> z(n, 0);
    bool any = false;
    for (int r = 0; r < n; r++)
      if (st[r].status == QCD_OK && etan[r] == 0.0) z[r] = 1, any = true;
    if (any) {
      QCD_TRY(upload_mask(z));
      QCD_TRY(blas_xmy(c, w.eta, w.eta, w.psi, QCD_PREC_F64, n, w.mask));
    }
  }

  // psi = 0 on entry for every active RHS (a solve without a starting guess):
  // the first true residual is eta itself (bit for bit eta - D 0), so the FP64
  // operator, whose rate on this GPU is 1/64 of FP32, is not applied
  bool psi_zero = true;
  {
    QCD_TRY(upload_mask(active));
    QCD_TRY(blas_norm2(c, w.psi, QCD_PREC_F64, n, w.rn2, w.mask));
    QCD_TRY(fetch(c, h_rn2, w.rn2, sizeof(double) * n));
    for (int r = 0; r < n; r++)
      if (active[r] && h_rn2[r] != 0.0) psi_zero = false;
  }
  bool first_residual = true;
  // D psi of the true residual in FP32 when every tolerance allows it
  bool resid_f32 = prec == QCD_PREC_F32 && P.resid_f32_tol > 0;
  for (int r = 0; r < n; r++)
    if (tol[r] < P.resid_f32_tol) resid_f32 = false;

  for (;;) {
    // true residual rho = eta - D psi (FP64 difference and norm)
    QCD_TRY(upload_mask(active));
    int nact_now = 0;
    for (int r = 0; r < n; r++) nact_now += active[r];
    if (first_residual && psi_zero) {
      QCD_TRY(blas_convert(c, w.eta, QCD_PREC_F64, w.rho, QCD_PREC_F64, n, w.mask));
    } else if (resid_f32) {
      // sapin and delta are free between restart cycles
      QCD_TRY(blas_convert(c, w.psi, QCD_PREC_F64, w.sapin, QCD_PREC_F32, n, w.mask));
      QCD_TRY(dslash_apply(c, w.sapin, w.delta, QCD_PREC_F32, n, 0, w.mask, nact_now));
      QCD_TRY(blas_convert(c, w.delta, QCD_PREC_F32, w.tmp, QCD_PREC_F64, n, w.mask));
      QCD_TRY(blas_xmy(c, w.eta, w.tmp, w.rho, QCD_PREC_F64, n, w.mask));
    } else {
      QCD_TRY(dslash_apply(c, w.psi, w.tmp, QCD_PREC_F64, n, 0, w.mask, nact_now));
      QCD_TRY(blas_xmy(c, w.eta, w.tmp, w.rho, QCD_PREC_F64, n, w.mask));
    }
    first_residual = false;
    QCD_TRY(blas_norm2(c, w.rho, QCD_PREC_F64, n, w.rn2, w.mask));
    QCD_TRY(fetch(c, h_rn2, w.rn2, sizeof(double) * n));
    int nact = 0;
    for (int r = 0; r < n; r++) {
      if (!active[r]) continue;
      double res = sqrt(h_rn2[r]) / etan[r];
      st[r].true_rel_residual = res;
      if (!isfinite(res)) {
        st[r].status = QCD_ERR_NONFINITE;
        active[r] = 0;
      } else if (res <= tol[r]) {
        active[r] = 0;
      } else if (st[r].outer_iters >= P.max_outer) {
        st[r].status = QCD_ERR_NOT_CONVERGED;
        active[r] = 0;
      } else {
        nact++;
        r0[r] = res;
        st[r].restarts++;
      }
    }
    if (nact == 0) break;

    // one restart cycle
    incyc = active;
    for (int r = 0; r < n; r++) kcount[r] = 0;
    int kmax = 0;
    for (int k = 0; k < nkv; k++) {
      QCD_TRY(upload_mask(incyc));
      int nin_now = 0;
      for (int r = 0; r < n; r++) nin_now += incyc[r];
      char* phik = w.phi + VI * k;
      char* chik = w.chi + VC * k;
      if (k == 0) QCD_TRY(blas_convert(c, w.rho, QCD_PREC_F64, w.rhoS, prec, n, w.mask));
      // SAP works in sapin; its first cycle reads the recursive residual rhoS
      if (use_dfl) {
        // deflated preconditioner: phi_k = Phi A^-1 Phi^+ rho + M_SAP(rho - D Phi A^-1 Phi^+ rho)
        QCD_TRY(dfl_low_mode(c, w.rhoS, phik, n, w.mask, nin_now, P.dfl_little_iters));
        QCD_TRY(dslash_apply(c, phik, w.delta, prec, n, 0, w.mask, nin_now));   // delta: scratch until the SAP
        QCD_TRY(blas_xmy(c, w.rhoS, w.delta, w.sapin, prec, n, w.mask));
        QCD_TRY(sap_apply(c, w.sapin, phik, w.delta, prec, n, w.mask, nin_now, 1));
      } else {
        QCD_TRY(sap_apply(c, w.sapin, phik, w.delta, prec, n, w.mask, nin_now, 0, w.rhoS));
      }
      QCD_TRY(dslash_apply(c, phik, chik, prec, n, 0, w.mask, nin_now, pchi));
      // Gram-Schmidt against chi_0..chi_{k-1}, normalisation, residual update;
      // the update also writes the next preconditioner input rhoS
      double2* ak = w.a + (size_t)k * nkv * n;
      QCD_TRY(blas_gs_dots(c, w.chi, pchi, VC, k, n, (double*)ak, w.mask, nin_now));
      // the recursive residual of the cycle is rhoS, in the inner precision
      QCD_TRY(blas_gs_orth(c, w.chi, pchi, VC, k, (const double*)ak, w.rhoS, prec, n, (double*)w.n2c, w.mask,
                           nin_now));
      {
        ProfScope ps(c, FAM_BLAS, 0.0, 0.0);
        k_gs_scalars<<<(n + 63) / 64, 64, 0, c->stream>>>(w.n2c, w.b + (size_t)k * n, w.inv, w.cc + (size_t)k * n, n,
                                                          w.mask);
      }
      QCD_CUDA_OK(cudaGetLastError());
      QCD_TRY(blas_gs_finish_inner(c, chik, pchi, w.inv, (const double*)(w.cc + (size_t)k * n), w.rhoS, prec, n,
                                   (double*)w.rn2c, w.mask, nin_now));
      QCD_TRY(fetch(c, h_rn2c, w.rn2c, sizeof(double2) * n));
      for (int r = 0; r < n; r++) h_rn2[r] = h_rn2c[r].x;
      kmax = k + 1;
      int nin = 0;
      for (int r = 0; r < n; r++) {
        if (!incyc[r]) continue;
        kcount[r] = k + 1;
        st[r].outer_iters++;
        double res = sqrt(h_rn2[r]) / etan[r];
        if (!isfinite(res) || res <= tol[r] || res <= P.restart_drop * r0[r] || st[r].outer_iters >= P.max_outer)
          incyc[r] = 0;
        else
          nin++;
      }
      if (nin == 0) break;
    }

    // back substitution and solution update
    QCD_TRY(fetch(c, h_a, w.a, sizeof(double2) * (size_t)nkv * nkv * n));
    QCD_TRY(fetch(c, h_b, w.b, sizeof(double) * (size_t)nkv * n));
    QCD_TRY(fetch(c, h_c, w.cc, sizeof(double2) * (size_t)nkv * n));
    for (int r = 0; r < n; r++) {
      for (int j = 0; j < nkv; j++) h_alpha[(size_t)j * n + r] = make_double2(0, 0);
      if (!active[r]) continue;
      const int m = kcount[r];
      for (int j = m - 1; j >= 0; j--) {
        double2 cj = h_c[(size_t)j * n + r];
        double sr = cj.x, si = cj.y;
        for (int i = j + 1; i < m; i++) {
          double2 aij = h_a[((size_t)i * nkv + j) * n + r];
          double2 al = h_alpha[(size_t)i * n + r];
          sr -= aij.x * al.x - aij.y * al.y;
          si -= aij.x * al.y + aij.y * al.x;
        }
        double bj = h_b[(size_t)j * n + r];
        if (!(bj > 0)) {
          st[r].status = QCD_ERR_BREAKDOWN;
          sr = si = 0;
          bj = 1;
        }
        h_alpha[(size_t)j * n + r] = make_double2(sr / bj, si / bj);
      }
    }
    QCD_CUDA_OK(cudaMemcpyAsync(w.alpha, h_alpha, sizeof(double2) * (size_t)nkv * n, cudaMemcpyHostToDevice,
                                c->stream));
    QCD_TRY(upload_mask(active));
    QCD_TRY(blas_multi_caxpy(c, w.psi, QCD_PREC_F64, w.phi, prec, kmax, VI, (const double*)w.alpha, 1.0, n,
                             w.mask));
    for (int r = 0; r < n; r++)
      if (active[r] && st[r].status == QCD_ERR_BREAKDOWN) active[r] = 0;
  }
  QCD_CUDA_OK(cudaStreamSynchronize(c->stream));
  return QCD_OK;
}

// Largest tile of right-hand sides that fits the device memory budget.
int solver_tile(qcd_ctx* c, int nrhs) {
  const qcd_solver_params& P = c->params;
  if (P.rhs_tile > 0) return P.rhs_tile < nrhs ? P.rhs_tile : nrhs;
  size_t freeb = 0, totalb = 0;
  cudaMemGetInfo(&freeb, &totalb);
  const int pchi = (P.precision == QCD_PREC_F32 && P.basis_half) ? QCD_PREC_H16 : P.precision;
  size_t per = 4 * spinor_bytes(c, QCD_PREC_F64) + ((size_t)P.nkv + 3) * spinor_bytes(c, P.precision) +
               (size_t)P.nkv * spinor_bytes(c, pchi);
  size_t budget = freeb > ((size_t)4 << 30) ? freeb - ((size_t)4 << 30) : freeb / 2;
  int t = (int)(budget / (per ? per : 1));
  if (t < 1) t = 1;
  if (t > 24) t = 24;
  return t < nrhs ? t : nrhs;
}
