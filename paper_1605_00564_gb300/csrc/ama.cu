// All-mode averaging of the nucleon two- and three-point functions
// (Sec. 2.1, eqs. caa1, caa2; Sec. 3, the fixed-iteration sloppy solves of
// Table 3), and the error model of eqs. ama1-ama3.
//
// qcd_ama_nucleon: for each of the N_G source positions g the 12 point
// sources are solved sloppily (to a tolerance, or with exactly N_iter GCR
// iterations), the two-point function is contracted and, with a sink
// separation, the sequential propagators through the sink are solved
// sloppily too (their own N_iter) and the three-point functions contracted;
// the first N_org positions are then solved to the exact tolerance (the
// point-source solve starting from its sloppy solution) and contracted
// again.  With Gaussian smearing set on the context (qcd_set_smearing) the
// point sources are smeared before the solves and the propagators' sink
// index after them (Sec. 2.3); the three-point functions then use the
// sink-smeared propagator for the sequential source and smear that source.
// The AMA estimate O_AMA = (1/N_org) sum_f [O^f - O_appx^f]
// + (1/N_G) sum_g O_appx^g is formed from the returned correlators.
#include <math.h>
#include <string.h>

#include <vector>

#include "qcd_internal.cuh"

qcd_status solver_run(qcd_ctx* c, int n, const double* tol, qcd_rhs_stats* st);
qcd_status contract_nucleon(qcd_ctx* c, const void* prop, int t0, double* corr_dev, int precision,
                            double2* partials);
qcd_status threept_internal(qcd_ctx* c, const void* S_int, const void* S_sink, const int src[4], int t_sep,
                            int direction, double tol, int n_iter, double* corr3, qcd_rhs_stats* st);

namespace {

__global__ void k_point12_at(double2* eta, int V, int site) {
  const int r = threadIdx.x;
  if (r < 12) eta[((size_t)r * 12 + r) * V + site] = make_double2(1.0, 0.0);
}

#define AMA_ARG(cond, ...)      \
  do {                          \
    if (!(cond)) {              \
      qcd_set_error(__VA_ARGS__); \
      return QCD_ERR_ARG;       \
    }                           \
  } while (0)

}  // namespace

extern "C" qcd_status qcd_ama_nucleon(qcd_ctx* c, const int* src, int n_src, const qcd_ama_params* p,
                                      double* c2_ama, double* c3_ama, double* c2_all, double* c3_all,
                                      qcd_rhs_stats* stats) {
  AMA_ARG(c && src && p && c2_ama, "null argument");
  if (!c->have_gauge) {
    qcd_set_error("no gauge field loaded");
    return QCD_ERR_STATE;
  }
  const int T = c->g.L[0];
  AMA_ARG(n_src >= 1 && p->n_exact >= 1 && p->n_exact <= n_src, "need 1 <= n_exact <= n_src");
  AMA_ARG(p->sloppy_tol > 0 && p->sloppy_tol < 1 && p->exact_tol > 0 && p->exact_tol < 1,
          "tolerances must be in (0, 1)");
  AMA_ARG(p->n_iter_2pt >= 0 && p->n_iter_3pt >= 0, "iteration counts must be >= 0");
  AMA_ARG(p->t_sep >= 0 && p->t_sep < T, "t_sep must be in [0, T)");
  AMA_ARG(p->t_sep == 0 || p->direction == 1 || p->direction == -1, "direction must be +1 or -1");
  AMA_ARG(p->t_sep == 0 || c3_ama, "c3_ama is needed with t_sep > 0");
  for (int i = 0; i < n_src; i++)
    for (int mu = 0; mu < 4; mu++) {
      const int x = src[4 * i + mu];
      AMA_ARG(x >= 0 && x < c->g.L[mu], "source %d outside the lattice", i);
      AMA_ARG(x % c->params.block[mu] == 0,
              "source %d is not a multiple of the SAP block extent in direction %d: the translation would not map "
              "the block decomposition onto itself", i, mu);
    }
  for (int i = 1; i < n_src; i++) {
    int par = 0;
    for (int mu = 0; mu < 4; mu++) par += (src[4 * i + mu] - src[mu]) / c->params.block[mu];
    AMA_ARG((par & 1) == 0,
            "sources 0 and %d differ by an odd number of blocks: the translation would exchange the SAP domains "
            "Omega and Omega*", i);
  }
  const int njobs = n_src + p->n_exact;
  const int per_job = 12 + (p->t_sep ? 24 : 0);
  std::vector<double> c2((size_t)njobs * 4 * T, 0.0), c3((size_t)njobs * 6 * T, 0.0);
  std::vector<qcd_rhs_stats> st((size_t)njobs * per_job);
  const size_t f64 = spinor_bytes(c, QCD_PREC_F64);
  const size_t prop_bytes = f64 * 12;
  QCD_TRY(devbuf_ensure(c->guess, prop_bytes * p->n_exact));
  const size_t npart = 2 * (size_t)c->g.V;
  const int basis_half = c->params.basis_half, max_outer = c->params.max_outer;
  qcd_status rc = QCD_OK;
  for (int j = 0; j < njobs && rc == QCD_OK; j++) {
    const bool exact = j >= n_src;
    const int si = exact ? j - n_src : j;
    const int* s = src + 4 * si;
    const int site = ((s[0] * c->g.L[3] + s[3]) * c->g.L[2] + s[2]) * c->g.L[1] + s[1];
    qcd_rhs_stats* sj = st.data() + (size_t)j * per_job;
    // forward propagator: wsD[0] = eta, wsD[1] = start
    if ((rc = devbuf_ensure(c->wsD[0], prop_bytes)) != QCD_OK) break;
    if ((rc = devbuf_ensure(c->wsD[1], prop_bytes)) != QCD_OK) break;
    if ((rc = devbuf_ensure(c->wsD[4], prop_bytes)) != QCD_OK) break;
    if (cudaMemsetAsync(c->wsD[0].p, 0, prop_bytes, c->stream) != cudaSuccess ||
        (exact ? cudaMemcpyAsync(c->wsD[1].p, (const char*)c->guess.p + prop_bytes * si, prop_bytes,
                                 cudaMemcpyDeviceToDevice, c->stream)
               : cudaMemsetAsync(c->wsD[1].p, 0, prop_bytes, c->stream)) != cudaSuccess) {
      qcd_set_error("source set-up failed");
      rc = QCD_ERR_CUDA;
      break;
    }
    k_point12_at<<<1, 32, 0, c->stream>>>((double2*)c->wsD[0].p, c->g.V, site);
    if (cudaGetLastError() != cudaSuccess) {
      qcd_set_error("point source launch failed");
      rc = QCD_ERR_CUDA;
      break;
    }
    if ((rc = smear_fields(c, c->wsD[0].p, 12)) != QCD_OK) break;      // smeared source
    const bool fixed = !exact && p->n_iter_2pt > 0;
    std::vector<double> tols(12, exact ? p->exact_tol : (fixed ? 1e-300 : p->sloppy_tol));
    if (exact) c->params.basis_half = 0;      // an FP16 Krylov basis serves the sloppy solves only
    if (fixed) c->params.max_outer = p->n_iter_2pt;
    rc = solver_run(c, 12, tols.data(), sj);
    c->params.basis_half = basis_half;
    c->params.max_outer = max_outer;
    if (rc != QCD_OK) break;
    if (fixed)
      for (int r = 0; r < 12; r++)
        if (sj[r].status == QCD_ERR_NOT_CONVERGED) sj[r].status = QCD_OK;   // stopped at N_iter by design
    // keep the propagator: the sloppy ones of the exact positions start the exact solves
    if (cudaMemcpyAsync(c->wsD[4].p, c->wsD[1].p, prop_bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess ||
        (!exact && si < p->n_exact &&
         cudaMemcpyAsync((char*)c->guess.p + prop_bytes * si, c->wsD[1].p, prop_bytes, cudaMemcpyDeviceToDevice,
                         c->stream) != cudaSuccess)) {
      qcd_set_error("propagator copy failed");
      rc = QCD_ERR_CUDA;
      break;
    }
    // the propagator seen at the sink: K S with a smeared sink
    const void* S_sink = c->wsD[4].p;
    if (c->smear_n > 0) {
      if ((rc = devbuf_ensure(c->smearbuf[1], prop_bytes)) != QCD_OK) break;
      if (cudaMemcpyAsync(c->smearbuf[1].p, c->wsD[4].p, prop_bytes, cudaMemcpyDeviceToDevice, c->stream) !=
          cudaSuccess) {
        qcd_set_error("propagator copy failed");
        rc = QCD_ERR_CUDA;
        break;
      }
      if ((rc = smear_fields(c, c->smearbuf[1].p, 12)) != QCD_OK) break;
      S_sink = c->smearbuf[1].p;
    }
    // two-point function
    if ((rc = devbuf_ensure(c->contract, sizeof(double2) * (npart + 2 * T))) != QCD_OK) break;
    double2* part = (double2*)c->contract.p;
    double2* cd = part + npart;
    const int prec = exact ? QCD_PREC_F64 : c->params.precision;
    if ((rc = contract_nucleon(c, S_sink, s[0], (double*)cd, prec, part)) != QCD_OK) break;
    if (cudaMemcpyAsync(c2.data() + (size_t)j * 4 * T, cd, sizeof(double2) * 2 * T, cudaMemcpyDeviceToHost,
                        c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess) {
      qcd_set_error("correlator copy failed");
      rc = QCD_ERR_CUDA;
      break;
    }
    // three-point functions
    if (p->t_sep) {
      if (exact) c->params.basis_half = 0;
      rc = threept_internal(c, c->wsD[4].p, S_sink, s, p->t_sep, p->direction,
                            exact ? p->exact_tol : p->sloppy_tol, exact ? 0 : p->n_iter_3pt,
                            c3.data() + (size_t)j * 6 * T, sj + 12);
      c->params.basis_half = basis_half;
      if (rc != QCD_OK) break;
    }
  }
  c->params.basis_half = basis_half;
  c->params.max_outer = max_outer;
  if (rc != QCD_OK) return rc;
  // O_AMA = (1/N_org) sum_f [O^f - O_appx^f] + (1/N_G) sum_g O_appx^g
  auto combine = [&](const std::vector<double>& all, int per, double* out) {
    for (int k = 0; k < per; k++) {
      double appx = 0, rest = 0;
      for (int g = 0; g < n_src; g++) appx += all[(size_t)g * per + k];
      for (int f = 0; f < p->n_exact; f++) rest += all[(size_t)(n_src + f) * per + k] - all[(size_t)f * per + k];
      out[k] = rest / p->n_exact + appx / n_src;
    }
  };
  combine(c2, 4 * T, c2_ama);
  if (p->t_sep) combine(c3, 6 * T, c3_ama);
  if (c2_all) memcpy(c2_all, c2.data(), sizeof(double) * c2.size());
  if (c3_all && p->t_sep) memcpy(c3_all, c3.data(), sizeof(double) * c3.size());
  qcd_status worst = QCD_OK;
  for (size_t r = 0; r < st.size(); r++) {
    if (stats) stats[r] = st[r];
    if (st[r].status != QCD_OK && worst == QCD_OK) worst = (qcd_status)st[r].status;
  }
  return worst;
}

// Error model of the AMA estimator (eqs. ama1-ama3) from measurements on
// n_conf configurations: exact[c][f], appx_org[c][f] (the sloppy observable
// at the same N_org positions), appx[c][g] (the sloppy observable at the N_G
// positions).  Covariances are sample covariances over the configurations.
//   Delta r = (1/N_org - 1/N_G) (1 - (1/N_org) sum_f corr(O^f, O_appx^f))
//   R       = (1/N_G^2) sum_{g != g'} corr(O_appx^g, O_appx^g')
//   model   = sqrt(1/N_G + 2 Delta r + R)          (sigma_AMA / sigma, eq. ama1)
//   measured = std_c(O_AMA) / sqrt(mean_f var_c(O^f))
extern "C" qcd_status qcd_ama_error_model(const double* exact, const double* appx_org, const double* appx,
                                          int n_conf, int n_org, int n_g, double* out) {
  if (!exact || !appx_org || !appx || !out) {
    qcd_set_error("null argument");
    return QCD_ERR_ARG;
  }
  if (n_conf < 2 || n_org < 1 || n_g < 1 || n_org > n_g) {
    qcd_set_error("need n_conf >= 2 and 1 <= n_org <= n_g");
    return QCD_ERR_ARG;
  }
  auto mean = [&](const double* a, int stride, int off) {
    double s = 0;
    for (int c = 0; c < n_conf; c++) s += a[(size_t)c * stride + off];
    return s / n_conf;
  };
  auto cov = [&](const double* a, int sa, int oa, const double* b, int sb, int ob) {
    const double ma = mean(a, sa, oa), mb = mean(b, sb, ob);
    double s = 0;
    for (int c = 0; c < n_conf; c++) s += (a[(size_t)c * sa + oa] - ma) * (b[(size_t)c * sb + ob] - mb);
    return s / (n_conf - 1);
  };
  double rho = 0, var_exact = 0;
  for (int f = 0; f < n_org; f++) {
    const double ve = cov(exact, n_org, f, exact, n_org, f), va = cov(appx_org, n_org, f, appx_org, n_org, f);
    if (!(ve > 0 && va > 0)) {
      qcd_set_error("a measurement has zero variance over the configurations");
      return QCD_ERR_ARG;
    }
    rho += cov(exact, n_org, f, appx_org, n_org, f) / sqrt(ve * va);
    var_exact += ve;
  }
  rho /= n_org;
  var_exact /= n_org;
  const double dr = (1.0 / n_org - 1.0 / n_g) * (1.0 - rho);
  double R = 0;
  for (int g = 0; g < n_g; g++)
    for (int h = 0; h < n_g; h++) {
      if (g == h) continue;
      const double vg = cov(appx, n_g, g, appx, n_g, g), vh = cov(appx, n_g, h, appx, n_g, h);
      if (!(vg > 0 && vh > 0)) {
        qcd_set_error("a measurement has zero variance over the configurations");
        return QCD_ERR_ARG;
      }
      R += cov(appx, n_g, g, appx, n_g, h) / sqrt(vg * vh);
    }
  R /= (double)n_g * n_g;
  // the AMA estimate on every configuration, and its spread
  std::vector<double> ama(n_conf);
  for (int c = 0; c < n_conf; c++) {
    double rest = 0, ap = 0;
    for (int f = 0; f < n_org; f++) rest += exact[(size_t)c * n_org + f] - appx_org[(size_t)c * n_org + f];
    for (int g = 0; g < n_g; g++) ap += appx[(size_t)c * n_g + g];
    ama[c] = rest / n_org + ap / n_g;
  }
  const double v_ama = cov(ama.data(), 1, 0, ama.data(), 1, 0);
  out[0] = dr;
  out[1] = R;
  const double m = 1.0 / n_g + 2.0 * dr + R;
  out[2] = m > 0 ? sqrt(m) : 0.0;
  out[3] = sqrt(v_ama / var_exact);
  return QCD_OK;
}
