// The extern "C" entry points declared in include/qcd.h.
#include <math.h>
#include <stdarg.h>
#include <stdlib.h>
#include <string.h>

#include <thread>
#include <vector>

#include "qcd_internal.cuh"

qcd_status solver_run(qcd_ctx* c, int n, const double* tol, qcd_rhs_stats* st);
int solver_tile(qcd_ctx* c, int nrhs);
qcd_status contract_nucleon(qcd_ctx* c, const void* prop, int t0, double* corr_dev, int precision,
                            double2* partials);

// --------------------------------------------------------------------------
// errors
// --------------------------------------------------------------------------
static thread_local char g_err[512];

void qcd_set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

#define ARG_CHECK(cond, ...)     \
  do {                           \
    if (!(cond)) {               \
      qcd_set_error(__VA_ARGS__); \
      return QCD_ERR_ARG;        \
    }                            \
  } while (0)

qcd_status devbuf_ensure(DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes) return QCD_OK;
  devbuf_free(b);
  cudaError_t e = cudaMalloc(&b.p, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    b.p = nullptr;
    cudaGetLastError();
    qcd_set_error("cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    return QCD_ERR_OOM;
  }
  b.bytes = bytes;
  return QCD_OK;
}

void devbuf_free(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

ProfScope::ProfScope(qcd_ctx* c_, int fam, double bytes, double flops, int kernels) : c(c_), idx(-1) {
  if (!c || !c->prof_on || c->prof_suspend) return;
  ProfRec r;
  r.fam = fam;
  r.kernels = kernels;
  r.bytes = bytes;
  r.flops = flops;
  for (cudaEvent_t* e : {&r.a, &r.b}) {
    if (!c->evpool.empty()) {
      *e = c->evpool.back();
      c->evpool.pop_back();
    } else if (cudaEventCreate(e) != cudaSuccess) {
      return;
    }
  }
  cudaEventRecord(r.a, c->stream);
  c->prof.push_back(r);
  idx = (int)c->prof.size() - 1;
}

ProfScope::~ProfScope() {
  if (idx >= 0) cudaEventRecord(c->prof[idx].b, c->stream);
}

static const char* kFamName[FAM_N] = {"dslash_f64", "dslash_f32", "sap_f64", "sap_f32", "blas",
                                      "layout",     "contract",   "deflation"};

namespace {

__global__ void k_point_sources(double2* eta, const int* site, int V, int n) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  int comp = r % 12;
  eta[((size_t)r * 12 + comp) * V + site[r]] = make_double2(1.0, 0.0);
}

qcd_status check_ready(qcd_ctx* c) {
  ARG_CHECK(c != nullptr, "null context");
  if (!c->have_gauge) {
    qcd_set_error("no gauge field loaded");
    return QCD_ERR_STATE;
  }
  return QCD_OK;
}

qcd_status validate_params(const qcd_ctx* c, const qcd_solver_params* p) {
  int vb = 1;
  for (int mu = 0; mu < 4; mu++) {
    int b = p->block[mu], L = c->g.L[mu];
    ARG_CHECK(b >= 1 && L % b == 0, "block extent %d does not divide lattice extent %d (direction %d)", b, L, mu);
    ARG_CHECK((L / b) % 2 == 0, "direction %d has an odd number (%d) of SAP blocks; the checkerboard needs an even one",
              mu, L / b);
    vb *= b;
  }
  ARG_CHECK(vb <= 1024, "SAP block volume %d exceeds 1024 sites", vb);
  ARG_CHECK(vb >= 32 && vb % 32 == 0, "SAP block volume %d must be a multiple of 32", vb);
  ARG_CHECK(p->ncy >= 1 && p->ncy <= 64, "ncy must be in [1, 64]");
  ARG_CHECK(p->nmr >= 1 && p->nmr <= 64, "nmr must be in [1, 64]");
  ARG_CHECK(p->nkv >= 1 && p->nkv <= 32, "nkv must be in [1, 32]");
  ARG_CHECK(p->max_outer >= 1, "max_outer must be >= 1");
  ARG_CHECK(p->restart_drop >= 0 && p->restart_drop < 1, "restart_drop must be in [0, 1)");
  ARG_CHECK(p->precision == QCD_PREC_F64 || p->precision == QCD_PREC_F32, "unknown precision %d", p->precision);
  ARG_CHECK(p->rhs_tile >= 0, "rhs_tile must be >= 0");
  ARG_CHECK(p->sap_half >= 0 && p->sap_half <= 2, "sap_half must be 0, 1 or 2");
  ARG_CHECK(p->dfl == 0 || p->dfl == 1, "dfl must be 0 or 1");
  ARG_CHECK(p->dfl_little_iters >= 1 && p->dfl_little_iters <= 64, "dfl_little_iters must be in [1, 64]");
  ARG_CHECK(p->dfl_gen_iters >= 0 && p->dfl_gen_iters <= 64, "dfl_gen_iters must be in [0, 64]");
  ARG_CHECK(p->graphs == 0 || p->graphs == 1, "graphs must be 0 or 1");
  ARG_CHECK(p->basis_half == 0 || p->basis_half == 1, "basis_half must be 0 or 1");
  ARG_CHECK(p->resid_f32_tol == 0 || (p->resid_f32_tol >= 1e-4 && p->resid_f32_tol < 1),
            "resid_f32_tol must be 0 or in [1e-4, 1)");
  return QCD_OK;
}

int site_index(const qcd_ctx* c, const int src[4]) {
  return ((src[0] * c->g.L[3] + src[3]) * c->g.L[2] + src[2]) * c->g.L[1] + src[1];
}

}  // namespace

extern "C" {

const char* qcd_status_string(qcd_status s) {
  switch (s) {
    case QCD_OK: return "ok";
    case QCD_ERR_ARG: return "invalid argument";
    case QCD_ERR_CUDA: return "CUDA error";
    case QCD_ERR_OOM: return "out of device memory";
    case QCD_ERR_NOT_CONVERGED: return "solver did not converge";
    case QCD_ERR_BREAKDOWN: return "solver breakdown";
    case QCD_ERR_NONFINITE: return "non-finite value";
    case QCD_ERR_TIMEOUT: return "device wait timed out";
    case QCD_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

const char* qcd_last_error(void) { return g_err; }

void qcd_default_params(qcd_solver_params* p) {
  if (!p) return;
  for (int mu = 0; mu < 4; mu++) p->block[mu] = 4;
  p->ncy = 5;
  p->nmr = 4;
  p->nkv = 16;
  p->max_outer = 2000;
  p->restart_drop = 1e-5;
  p->precision = QCD_PREC_F32;
  p->rhs_tile = 0;
  p->sap_half = 0;
  p->dfl = 1;
  p->dfl_little_iters = 16;
  p->dfl_gen_iters = 0;
  p->graphs = 1;
  p->basis_half = 0;
  p->resid_f32_tol = 0;
}

qcd_status qcd_create(qcd_ctx** out, const int dims[4], void* cuda_stream) {
  ARG_CHECK(out != nullptr && dims != nullptr, "null argument");
  *out = nullptr;
  long long V = 1;
  for (int i = 0; i < 4; i++) {
    ARG_CHECK(dims[i] >= 2, "lattice extent %d must be >= 2", dims[i]);
    V *= dims[i];
  }
  ARG_CHECK(V < (1LL << 31), "lattice volume too large");
  qcd_ctx* c = new qcd_ctx();
  for (int i = 0; i < 4; i++) c->dims[i] = dims[i];
  // dims = {T, X, Y, Z}; direction mu: 0 t, 1 x, 2 y, 3 z
  for (int mu = 0; mu < 4; mu++) c->g.L[mu] = dims[mu];
  c->g.V = (int)V;
  c->g.stride[1] = 1;
  c->g.stride[2] = dims[1];
  c->g.stride[3] = dims[1] * dims[2];
  c->g.stride[0] = dims[1] * dims[2] * dims[3];
  c->g.bc_t = -1;
  c->stream = (cudaStream_t)cuda_stream;
  qcd_default_params(&c->params);
  if (validate_params(c, &c->params) != QCD_OK) {
    // default 4^4 blocks do not fit this lattice: fall back to 2^4 where possible
    for (int mu = 0; mu < 4; mu++) c->params.block[mu] = 2;
  }
  *out = c;
  return QCD_OK;
}

void qcd_destroy(qcd_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  devbuf_free(c->gaugeD);
  devbuf_free(c->gaugeF);
  devbuf_free(c->cloverD);
  devbuf_free(c->cloverF);
  devbuf_free(c->gaugeH);
  devbuf_free(c->cloverH);
  for (int i = 0; i < 8; i++) {
    devbuf_free(c->wsD[i]);
    devbuf_free(c->wsF[i]);
  }
  devbuf_free(c->basisF);
  devbuf_free(c->basisD);
  devbuf_free(c->red);
  devbuf_free(c->scal);
  devbuf_free(c->contract);
  devbuf_free(c->stage);
  devbuf_free(c->guess);
  devbuf_free(c->small);
  devbuf_free(c->gaugeS);
  devbuf_free(c->smearbuf[0]);
  devbuf_free(c->smearbuf[1]);
  if (c->host_scal) cudaFreeHost(c->host_scal);
  dfl_free(c);
  for (auto& gph : c->sap_graphs) cudaGraphExecDestroy(gph.exec);
  for (auto& r : c->prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : c->evpool) cudaEventDestroy(e);
  delete c;
}

qcd_status qcd_load_gauge(qcd_ctx* c, const double* U, int U_on_device, double csw, double kappa, int time_bc) {
  ARG_CHECK(c != nullptr && U != nullptr, "null argument");
  ARG_CHECK(time_bc == 1 || time_bc == -1, "time_bc must be +1 or -1");
  ARG_CHECK(isfinite(csw) && isfinite(kappa), "non-finite csw or kappa");
  c->g.bc_t = time_bc;
  c->kappa = kappa;
  c->csw = csw;
  const size_t bytes = (size_t)c->g.V * 4 * 9 * sizeof(double2);
  const double* Ud = U;
  if (!U_on_device) {
    QCD_TRY(devbuf_ensure(c->stage, bytes));
    QCD_CUDA_OK(cudaMemcpyAsync(c->stage.p, U, bytes, cudaMemcpyHostToDevice, c->stream));
    Ud = (const double*)c->stage.p;
  }
  QCD_TRY(layout_gauge_import(c, Ud));
  QCD_TRY(layout_clover_build(c));
  QCD_CUDA_OK(cudaStreamSynchronize(c->stream));
  c->have_gauge = 1;
  return QCD_OK;
}

qcd_status qcd_set_params(qcd_ctx* c, const qcd_solver_params* p) {
  ARG_CHECK(c != nullptr && p != nullptr, "null argument");
  QCD_TRY(validate_params(c, p));
  bool same_blocks = true;
  for (int mu = 0; mu < 4; mu++) same_blocks = same_blocks && p->block[mu] == c->params.block[mu];
  if (!same_blocks) dfl_free(c);
  c->params = *p;
  return QCD_OK;
}

qcd_status qcd_apply_dirac(qcd_ctx* c, const double* in, double* out, int nrhs, int dagger, int precision) {
  QCD_TRY(check_ready(c));
  ARG_CHECK(in && out && in != out, "in and out must be distinct non-null device pointers");
  ARG_CHECK(nrhs >= 1, "nrhs must be >= 1");
  ARG_CHECK(precision == QCD_PREC_F64 || precision == QCD_PREC_F32, "unknown precision");
  const size_t b = spinor_bytes(c, precision) * nrhs;
  DevBuf* ws = precision == QCD_PREC_F64 ? c->wsD : c->wsF;
  QCD_TRY(devbuf_ensure(ws[4], b));
  QCD_TRY(devbuf_ensure(ws[5], b));
  QCD_TRY(layout_spinor_import(c, in, ws[4].p, precision, nrhs));
  QCD_TRY(dslash_apply(c, ws[4].p, ws[5].p, precision, nrhs, dagger ? 1 : 0, nullptr, nrhs));
  QCD_TRY(layout_spinor_export(c, ws[5].p, out, precision, nrhs));
  QCD_CUDA_OK(cudaStreamSynchronize(c->stream));
  return QCD_OK;
}

qcd_status qcd_apply_sap(qcd_ctx* c, const double* eta, double* psi, int nrhs, int precision) {
  QCD_TRY(check_ready(c));
  ARG_CHECK(eta && psi && eta != psi, "eta and psi must be distinct non-null device pointers");
  ARG_CHECK(nrhs >= 1, "nrhs must be >= 1");
  ARG_CHECK(precision == QCD_PREC_F64 || precision == QCD_PREC_F32, "unknown precision");
  const size_t b = spinor_bytes(c, precision) * nrhs;
  DevBuf* ws = precision == QCD_PREC_F64 ? c->wsD : c->wsF;
  QCD_TRY(devbuf_ensure(ws[4], b));
  QCD_TRY(devbuf_ensure(ws[5], b));
  QCD_TRY(devbuf_ensure(ws[6], b));
  QCD_TRY(layout_spinor_import(c, eta, ws[4].p, precision, nrhs));
  QCD_TRY(sap_apply(c, ws[4].p, ws[5].p, ws[6].p, precision, nrhs, nullptr, nrhs));
  QCD_TRY(layout_spinor_export(c, ws[5].p, psi, precision, nrhs));
  QCD_CUDA_OK(cudaStreamSynchronize(c->stream));
  return QCD_OK;
}

qcd_status qcd_solve(qcd_ctx* c, const double* eta, double* psi, int nrhs, const double* rel_tol,
                     qcd_rhs_stats* stats) {
  QCD_TRY(check_ready(c));
  ARG_CHECK(eta && psi && rel_tol && eta != psi, "eta, psi, rel_tol must be non-null; eta != psi");
  ARG_CHECK(nrhs >= 1, "nrhs must be >= 1");
  for (int r = 0; r < nrhs; r++) ARG_CHECK(rel_tol[r] > 0 && rel_tol[r] < 1, "rel_tol[%d] must be in (0, 1)", r);
  std::vector<qcd_rhs_stats> st(nrhs);
  const int tile = solver_tile(c, nrhs);
  const size_t per = (size_t)c->g.V * 24;   // doubles of one canonical spinor
  for (int r0 = 0; r0 < nrhs; r0 += tile) {
    int n = nrhs - r0 < tile ? nrhs - r0 : tile;
    QCD_TRY(devbuf_ensure(c->wsD[0], spinor_bytes(c, QCD_PREC_F64) * n));
    QCD_TRY(devbuf_ensure(c->wsD[1], spinor_bytes(c, QCD_PREC_F64) * n));
    QCD_TRY(layout_spinor_import(c, eta + per * r0, c->wsD[0].p, QCD_PREC_F64, n));
    QCD_TRY(layout_spinor_import(c, psi + per * r0, c->wsD[1].p, QCD_PREC_F64, n));
    QCD_TRY(solver_run(c, n, rel_tol + r0, st.data() + r0));
    QCD_TRY(layout_spinor_export(c, c->wsD[1].p, psi + per * r0, QCD_PREC_F64, n));
  }
  QCD_CUDA_OK(cudaStreamSynchronize(c->stream));
  qcd_status worst = QCD_OK;
  int nbad = 0;
  for (int r = 0; r < nrhs; r++) {
    if (stats) stats[r] = st[r];
    if (st[r].status != QCD_OK) {
      nbad++;
      if (worst == QCD_OK) worst = (qcd_status)st[r].status;
    }
  }
  if (worst != QCD_OK) qcd_set_error("%d of %d right-hand sides did not converge", nbad, nrhs);
  return worst;
}

qcd_status qcd_solve_multi(qcd_ctx* const* ctxs, int nctx, const double* const* eta, double* const* psi,
                           const int* nrhs, const double* const* rel_tol, qcd_rhs_stats* const* stats) {
  ARG_CHECK(ctxs && nctx >= 1 && eta && psi && nrhs && rel_tol, "null argument");
  for (int i = 0; i < nctx; i++) {
    QCD_TRY(check_ready(ctxs[i]));
    for (int j = 0; j < i; j++)
      ARG_CHECK(ctxs[j] != ctxs[i], "context %d appears twice", i);
    ARG_CHECK(nctx == 1 || ctxs[i]->stream != nullptr,
              "qcd_solve_multi needs a non-default stream per context to run the lattices concurrently");
  }
  std::vector<qcd_status> rc(nctx, QCD_OK);
  std::vector<std::thread> th;
  int dev = 0;
  QCD_CUDA_OK(cudaGetDevice(&dev));
  for (int i = 0; i < nctx; i++)
    th.emplace_back([&, i]() {
      cudaSetDevice(dev);
      rc[i] = qcd_solve(ctxs[i], eta[i], psi[i], nrhs[i], rel_tol[i], stats ? stats[i] : nullptr);
    });
  for (auto& t : th) t.join();
  for (int i = 0; i < nctx; i++)
    if (rc[i] != QCD_OK) return rc[i];
  return QCD_OK;
}

qcd_status qcd_nucleon_2pt(qcd_ctx* c, const double* prop, const int src[4], double* corr, int precision) {
  QCD_TRY(check_ready(c));
  ARG_CHECK(prop && src && corr, "null argument");
  ARG_CHECK(precision == QCD_PREC_F64 || precision == QCD_PREC_F32, "unknown precision");
  for (int mu = 0; mu < 4; mu++) ARG_CHECK(src[mu] >= 0 && src[mu] < c->g.L[mu], "source outside the lattice");
  const int T = c->g.L[0];
  QCD_TRY(devbuf_ensure(c->wsD[4], spinor_bytes(c, QCD_PREC_F64) * 12));
  QCD_TRY(layout_spinor_import(c, prop, c->wsD[4].p, QCD_PREC_F64, 12));
  const size_t npart = 2 * (size_t)c->g.V;   // >= 2 * (V / sites per CTA)
  QCD_TRY(devbuf_ensure(c->contract, sizeof(double2) * (npart + 2 * T)));
  double2* part = (double2*)c->contract.p;
  double2* cd = part + npart;
  QCD_TRY(contract_nucleon(c, c->wsD[4].p, src[0], (double*)cd, precision, part));
  QCD_CUDA_OK(cudaMemcpyAsync(corr, cd, sizeof(double2) * 2 * T, cudaMemcpyDeviceToHost, c->stream));
  QCD_CUDA_OK(cudaStreamSynchronize(c->stream));
  return QCD_OK;
}

qcd_status qcd_ama_nucleon_2pt(qcd_ctx* c, const int* src, int n_src, int n_exact, double sloppy_tol,
                               double exact_tol, double* corr_ama, double* corr_all, qcd_rhs_stats* stats) {
  QCD_TRY(check_ready(c));
  ARG_CHECK(src && corr_ama, "null argument");
  ARG_CHECK(n_src >= 1 && n_exact >= 1 && n_exact <= n_src, "need 1 <= n_exact <= n_src");
  ARG_CHECK(sloppy_tol > 0 && sloppy_tol < 1 && exact_tol > 0 && exact_tol < 1, "tolerances must be in (0, 1)");
  for (int i = 0; i < n_src; i++)
    for (int mu = 0; mu < 4; mu++) {
      int x = src[4 * i + mu];
      ARG_CHECK(x >= 0 && x < c->g.L[mu], "source %d outside the lattice", i);
      ARG_CHECK(x % c->params.block[mu] == 0,
                "source %d is not a multiple of the SAP block extent in direction %d: the translation would not map "
                "the block decomposition onto itself", i, mu);
    }
  // the translations between the sources must map Omega onto Omega (even shift in blocks)
  for (int i = 1; i < n_src; i++) {
    int par = 0;
    for (int mu = 0; mu < 4; mu++) par += (src[4 * i + mu] - src[mu]) / c->params.block[mu];
    ARG_CHECK((par & 1) == 0,
              "sources 0 and %d differ by an odd number of blocks: the translation would exchange the SAP domains "
              "Omega and Omega*", i);
  }
  const int T = c->g.L[0];
  const int njobs = n_src + n_exact;   // sloppy solves of every source, then exact solves
  std::vector<double> corr((size_t)njobs * 4 * T);
  std::vector<qcd_rhs_stats> st((size_t)njobs * 12);
  int tile = solver_tile(c, 12 * njobs);
  int spt = tile / 12 > 0 ? tile / 12 : 1;   // sources per tile
  const size_t npart = 2 * (size_t)c->g.V;
  QCD_TRY(devbuf_ensure(c->contract, sizeof(double2) * (npart + 2 * T)));
  double2* part = (double2*)c->contract.p;
  double2* cd = part + npart;
  std::vector<int> sites(12 * spt);
  std::vector<double> tols(12 * spt);
  // the source sites live in a context workspace (no allocation once it is large enough)
  QCD_TRY(devbuf_ensure(c->small, sizeof(int) * 12 * spt));
  int* d_sites = (int*)c->small.p;
  DevBuf& guess = c->guess;   // sloppy propagators of the exact-solve sources
  QCD_TRY(devbuf_ensure(guess, spinor_bytes(c, QCD_PREC_F64) * 12 * n_exact));
  qcd_status rc = QCD_OK;
  for (int j0 = 0; j0 < njobs && rc == QCD_OK; j0 += spt) {
    // jobs of one tile share a tolerance: do not mix sloppy and exact
    int nj = 0;
    while (j0 + nj < njobs && nj < spt && ((j0 + nj < n_src) == (j0 < n_src))) nj++;
    const double tol = j0 < n_src ? sloppy_tol : exact_tol;
    const int n = 12 * nj;
    for (int k = 0; k < nj; k++) {
      int si = (j0 + k) < n_src ? (j0 + k) : (j0 + k - n_src);
      for (int r = 0; r < 12; r++) {
        sites[12 * k + r] = site_index(c, src + 4 * si);
        tols[12 * k + r] = tol;
      }
    }
    const size_t b = spinor_bytes(c, QCD_PREC_F64) * n;
    if ((rc = devbuf_ensure(c->wsD[0], b)) != QCD_OK) break;
    if ((rc = devbuf_ensure(c->wsD[1], b)) != QCD_OK) break;
    if (cudaMemsetAsync(c->wsD[0].p, 0, b, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->wsD[1].p, 0, b, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(d_sites, sites.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
      rc = QCD_ERR_CUDA;
      qcd_set_error("source set-up failed");
      break;
    }
    // the exact solve of a source starts from that source's sloppy solution
    const size_t prop_bytes = spinor_bytes(c, QCD_PREC_F64) * 12;
    if (j0 >= n_src)
      for (int k = 0; k < nj; k++)
        if (cudaMemcpyAsync((char*)c->wsD[1].p + prop_bytes * k, (const char*)guess.p + prop_bytes * (j0 + k - n_src),
                            prop_bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess) {
          rc = QCD_ERR_CUDA;
          qcd_set_error("initial guess copy failed");
        }
    if (rc != QCD_OK) break;
    {
      ProfScope ps(c, FAM_LAYOUT, 0.0, 0.0);
      k_point_sources<<<(n + 63) / 64, 64, 0, c->stream>>>((double2*)c->wsD[0].p, d_sites, c->g.V, n);
    }
    // an FP16 Krylov basis (basis_half) serves the sloppy tiles only
    const int basis_half = c->params.basis_half;
    if (j0 >= n_src) c->params.basis_half = 0;
    rc = solver_run(c, n, tols.data(), st.data() + (size_t)12 * j0);
    c->params.basis_half = basis_half;
    if (rc != QCD_OK) break;
    if (j0 < n_src)
      for (int k = 0; k < nj; k++)
        if (j0 + k < n_exact &&
            cudaMemcpyAsync((char*)guess.p + prop_bytes * (j0 + k), (const char*)c->wsD[1].p + prop_bytes * k,
                            prop_bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess) {
          rc = QCD_ERR_CUDA;
          qcd_set_error("initial guess copy failed");
        }
    if (rc != QCD_OK) break;
    for (int k = 0; k < nj && rc == QCD_OK; k++) {
      int si = (j0 + k) < n_src ? (j0 + k) : (j0 + k - n_src);
      const char* prop = (const char*)c->wsD[1].p + spinor_bytes(c, QCD_PREC_F64) * 12 * k;
      int prec = j0 < n_src ? c->params.precision : QCD_PREC_F64;
      rc = contract_nucleon(c, prop, src[4 * si], (double*)cd, prec, part);
      if (rc != QCD_OK) break;
      if (cudaMemcpyAsync(corr.data() + (size_t)(j0 + k) * 4 * T, cd, sizeof(double2) * 2 * T,
                          cudaMemcpyDeviceToHost, c->stream) != cudaSuccess) {
        rc = QCD_ERR_CUDA;
        break;
      }
    }
  }
  cudaStreamSynchronize(c->stream);
  if (rc != QCD_OK) return rc;
  // O_AMA = (1/N_org) sum_f [O^f - O_appx^f] + (1/N_G) sum_g O_appx^g
  for (int k = 0; k < 4 * T; k++) {
    double appx = 0, rest = 0;
    for (int g = 0; g < n_src; g++) appx += corr[(size_t)g * 4 * T + k];
    for (int f = 0; f < n_exact; f++) rest += corr[(size_t)(n_src + f) * 4 * T + k] - corr[(size_t)f * 4 * T + k];
    corr_ama[k] = rest / n_exact + appx / n_src;
  }
  if (corr_all) memcpy(corr_all, corr.data(), sizeof(double) * corr.size());
  qcd_status worst = QCD_OK;
  for (size_t r = 0; r < st.size(); r++) {
    if (stats) stats[r] = st[r];
    if (st[r].status != QCD_OK && worst == QCD_OK) worst = (qcd_status)st[r].status;
  }
  return worst;
}

qcd_status qcd_profile_enable(qcd_ctx* c, int on) {
  ARG_CHECK(c != nullptr, "null context");
  QCD_CUDA_OK(cudaStreamSynchronize(c->stream));
  for (auto& r : c->prof) {
    c->evpool.push_back(r.a);
    c->evpool.push_back(r.b);
  }
  c->prof.clear();
  c->prof_on = on ? 1 : 0;
  return QCD_OK;
}

qcd_status qcd_profile_read(qcd_ctx* c, qcd_kernel_time* out, int max, int* n) {
  ARG_CHECK(c != nullptr && out != nullptr && n != nullptr, "null argument");
  QCD_CUDA_OK(cudaStreamSynchronize(c->stream));
  qcd_kernel_time acc[FAM_N];
  memset(acc, 0, sizeof(acc));
  for (auto& r : c->prof) {
    float ms = 0;
    QCD_CUDA_OK(cudaEventElapsedTime(&ms, r.a, r.b));
    acc[r.fam].launches += r.kernels;
    acc[r.fam].ms += ms;
    acc[r.fam].bytes += r.bytes;
    acc[r.fam].flops += r.flops;
    c->evpool.push_back(r.a);
    c->evpool.push_back(r.b);
  }
  c->prof.clear();
  int k = 0;
  for (int f = 0; f < FAM_N && k < max; f++) {
    if (!acc[f].launches) continue;
    out[k] = acc[f];
    snprintf(out[k].name, sizeof(out[k].name), "%s", kFamName[f]);
    k++;
  }
  *n = k;
  return QCD_OK;
}

qcd_status qcd_deflation_setup(qcd_ctx* c, const double* init, int ns, int n_inv) {
  QCD_TRY(check_ready(c));
  ARG_CHECK(init != nullptr, "null argument");
  ARG_CHECK(ns >= 1 && ns <= 32, "ns must be in [1, 32]");
  ARG_CHECK(n_inv >= 0 && n_inv <= 32, "n_inv must be in [0, 32]");
  for (int mu = 0; mu < 4; mu++)
    ARG_CHECK(c->params.block[mu] >= 2, "deflation needs block extents >= 2 (direction %d)", mu);
  QCD_TRY(dfl_setup(c, init, ns, n_inv));
  QCD_CUDA_OK(cudaStreamSynchronize(c->stream));
  return QCD_OK;
}

qcd_status qcd_deflation_fields(qcd_ctx* c, double* out) {
  QCD_TRY(check_ready(c));
  ARG_CHECK(out != nullptr, "null argument");
  if (!dfl_ready(c)) {
    qcd_set_error("no deflation subspace");
    return QCD_ERR_STATE;
  }
  QCD_TRY(layout_spinor_export(c, dfl_phi(c), out, QCD_PREC_F32, dfl_ns(c)));
  QCD_CUDA_OK(cudaStreamSynchronize(c->stream));
  return QCD_OK;
}

qcd_status qcd_deflation_little_matrix(qcd_ctx* c, double* out) {
  QCD_TRY(check_ready(c));
  ARG_CHECK(out != nullptr, "null argument");
  if (!dfl_ready(c)) {
    qcd_set_error("no deflation subspace");
    return QCD_ERR_STATE;
  }
  const size_t n = (size_t)dfl_nblk(c) * 9 * dfl_ns(c) * dfl_ns(c);
  // A is stored in FP64: copy it out as it is
  QCD_CUDA_OK(cudaMemcpyAsync(out, dfl_little(c), sizeof(double2) * n, cudaMemcpyDeviceToHost, c->stream));
  QCD_CUDA_OK(cudaStreamSynchronize(c->stream));
  return QCD_OK;
}

qcd_status qcd_deflation_little(qcd_ctx* c, const double* in, double* out, int n, int mode, int m) {
  QCD_TRY(check_ready(c));
  ARG_CHECK(in && out && n >= 1, "bad argument");
  ARG_CHECK(mode == 0 || mode == 1, "mode must be 0 or 1");
  ARG_CHECK(m >= 1 && m <= 64, "m must be in [1, 64]");
  if (!dfl_ready(c)) {
    qcd_set_error("no deflation subspace");
    return QCD_ERR_STATE;
  }
  return dfl_little_host(c, in, out, n, mode, m);
}

qcd_status qcd_get_clover(qcd_ctx* c, double* out) {
  QCD_TRY(check_ready(c));
  ARG_CHECK(out != nullptr, "null argument");
  QCD_TRY(clover_export(c, out));
  QCD_CUDA_OK(cudaStreamSynchronize(c->stream));
  return QCD_OK;
}

}  // extern "C"
