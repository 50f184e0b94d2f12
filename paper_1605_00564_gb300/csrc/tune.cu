// Autotuner of the implementation parameters of the solver: SAP block shape,
// 16-bit or 32-bit block copies in the SAP kernel, GCR restart length and the
// number of right-hand sides solved together.  The method's own parameters
// (n_cy, n_mr, tolerances, deflation) are left as the caller set them.
//
// Each candidate solves the caller's right-hand sides to the given tolerance
// (time to solution, CUDA events on the context's stream); the fastest
// candidate that converged is kept.  Results are cached in a text file, one
// line per key: lattice, couplings, boundary condition, precision, tolerance,
// number of RHS and GPU name.
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "qcd_internal.cuh"

namespace {

std::string tune_key(qcd_ctx* c, int nrhs, double tol) {
  cudaDeviceProp prop;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaGetDeviceProperties(&prop, dev);
  char buf[512];
  snprintf(buf, sizeof(buf),
           "%dx%dx%dx%d k=%.6f csw=%.4f bc=%d prec=%d bh=%d ncy=%d nmr=%d dfl=%d tol=%.1e n=%d gpu=%s", c->dims[0],
           c->dims[1], c->dims[2], c->dims[3], c->kappa, c->csw, c->g.bc_t, c->params.precision,
           c->params.basis_half, c->params.ncy, c->params.nmr, c->params.dfl, tol, nrhs, prop.name);
  for (char* p = buf; *p; p++)
    if (*p == '|' || *p == '\n') *p = '_';
  return buf;
}

bool cache_lookup(const char* path, const std::string& key, qcd_solver_params* p) {
  if (!path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[1024];
  bool found = false;
  while (fgets(line, sizeof(line), f)) {
    char* bar = strchr(line, '|');
    if (!bar) continue;
    *bar = 0;
    if (key != line) continue;
    int b0, b1, b2, b3, half, nkv, tile;
    if (sscanf(bar + 1, " block=%d,%d,%d,%d sap_half=%d nkv=%d rhs_tile=%d", &b0, &b1, &b2, &b3, &half, &nkv,
               &tile) == 7) {
      p->block[0] = b0; p->block[1] = b1; p->block[2] = b2; p->block[3] = b3;
      p->sap_half = half;
      p->nkv = nkv;
      p->rhs_tile = tile;
      found = true;   // the last matching line wins
    }
  }
  fclose(f);
  return found;
}

void cache_store(const char* path, const std::string& key, const qcd_solver_params& p, float ms) {
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s| block=%d,%d,%d,%d sap_half=%d nkv=%d rhs_tile=%d ms=%.1f\n", key.c_str(), p.block[0], p.block[1],
          p.block[2], p.block[3], p.sap_half, p.nkv, p.rhs_tile, ms);
  fclose(f);
}

bool block_ok(const qcd_ctx* c, const int b[4]) {
  int vb = 1;
  for (int mu = 0; mu < 4; mu++) {
    if (b[mu] < 1 || c->g.L[mu] % b[mu] || (c->g.L[mu] / b[mu]) % 2) return false;
    vb *= b[mu];
  }
  return vb >= 32 && vb <= 1024 && vb % 32 == 0;
}

}  // namespace

extern "C" qcd_status qcd_autotune(qcd_ctx* c, const double* eta, int nrhs, double tol, const char* cache_path,
                                   qcd_solver_params* best) {
  if (!c || !eta || nrhs < 1 || !(tol > 0 && tol < 1)) {
    qcd_set_error("bad argument");
    return QCD_ERR_ARG;
  }
  if (!c->have_gauge) {
    qcd_set_error("no gauge field loaded");
    return QCD_ERR_STATE;
  }
  const std::string key = tune_key(c, nrhs, tol);
  qcd_solver_params p = c->params;
  if (cache_lookup(cache_path, key, &p)) {
    QCD_TRY(qcd_set_params(c, &p));
    if (best) *best = c->params;
    return QCD_OK;
  }
  const qcd_solver_params base = c->params;
  std::vector<qcd_solver_params> cand;
  const int blocks[][4] = {{base.block[0], base.block[1], base.block[2], base.block[3]},
                           {4, 4, 4, 4}, {8, 4, 4, 4}, {4, 4, 4, 8}, {4, 8, 4, 4}};
  for (const auto& b : blocks) {
    if (!block_ok(c, b)) continue;
    bool dup = false;
    for (const auto& q : cand) dup = dup || (memcmp(q.block, b, sizeof(q.block)) == 0);
    if (dup) continue;
    for (int half = 0; half < 2; half++)
      for (int nkv : {16, 32})
        for (int tile : {nrhs, (nrhs + 1) / 2}) {
          qcd_solver_params q = base;
          memcpy(q.block, b, sizeof(q.block));
          q.sap_half = half;
          q.nkv = nkv;
          q.rhs_tile = tile;
          cand.push_back(q);
        }
  }
  const size_t bytes = (size_t)c->g.V * 24 * sizeof(double) * nrhs;
  double* psi = nullptr;
  QCD_CUDA_OK(cudaMalloc((void**)&psi, bytes));
  std::vector<double> tols(nrhs, tol);
  std::vector<qcd_rhs_stats> st(nrhs);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best_ms = -1;
  qcd_solver_params best_p = base;
  qcd_status rc = QCD_OK;
  for (const auto& q : cand) {
    if ((rc = qcd_set_params(c, &q)) != QCD_OK) break;
    cudaMemsetAsync(psi, 0, bytes, c->stream);
    cudaEventRecord(e0, c->stream);
    qcd_status s = qcd_solve(c, eta, psi, nrhs, tols.data(), st.data());
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (s == QCD_OK && (best_ms < 0 || ms < best_ms)) {
      best_ms = ms;
      best_p = c->params;
    } else if (s != QCD_OK && s != QCD_ERR_NOT_CONVERGED) {
      rc = s;
      break;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(psi);
  if (rc != QCD_OK) {
    qcd_set_params(c, &base);
    return rc;
  }
  if (best_ms < 0) {
    qcd_set_params(c, &base);
    qcd_set_error("no candidate converged");
    return QCD_ERR_NOT_CONVERGED;
  }
  QCD_TRY(qcd_set_params(c, &best_p));
  cache_store(cache_path, key, best_p, best_ms);
  if (best) *best = c->params;
  return QCD_OK;
}
