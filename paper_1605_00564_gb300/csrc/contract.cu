// Nucleon two-point function (eq. Nop and the P+- projections of Sec. 2.3)
// on a propagator in the internal FP64 spinor layout; the kernels and the
// contraction formulas are in nucleon_kernels.cuh.
#include "nucleon_kernels.cuh"

int contract_sites_per_cta(const qcd_ctx* c) {
  return nucleon::sites_per_cta((long long)c->g.L[1] * c->g.L[2] * c->g.L[3]);
}

// corr_dev: [2][T] double2.  prop: 12 FP64 internal spinors (rhs = 3 spin + colour).
// partials: at least 2 V / ns double2.
qcd_status contract_nucleon(qcd_ctx* c, const void* prop, int t0, double* corr_dev, int precision,
                            double2* partials) {
  const int ns = contract_sites_per_cta(c);
  const int nb = c->g.V / ns;
  const int T = c->g.L[0];
  const int per_t = nb / T;
  const int bc3 = c->g.bc_t * c->g.bc_t * c->g.bc_t;
  const int threads = nucleon::cta_threads(ns);
  // algorithmic cost per site: the 144 complex propagator entries read once;
  // 36 colour-permutation pairs x (16 + 64 + 32) complex multiply-adds
  ProfScope ps(c, FAM_CONTRACT, (double)c->g.V * 144 * 16, (double)c->g.V * 36 * 112 * 8, 2);
  if (precision == QCD_PREC_F64) {
    const size_t smem = (size_t)144 * ns * sizeof(Cplx<double>);
    QCD_CUDA_OK(cudaFuncSetAttribute(nucleon::k_sites<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    nucleon::k_sites<double, false><<<nb, threads, smem, c->stream>>>((const double2*)prop, c->g.V, ns, partials);
  } else {
    const size_t smem = (size_t)144 * ns * sizeof(Cplx<float>);
    QCD_CUDA_OK(cudaFuncSetAttribute(nucleon::k_sites<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    nucleon::k_sites<float, false><<<nb, threads, smem, c->stream>>>((const double2*)prop, c->g.V, ns, partials);
  }
  QCD_CUDA_OK(cudaGetLastError());
  nucleon::k_timeslices<<<T, 256, 0, c->stream>>>(partials, per_t, T, t0, bc3, (double2*)corr_dev);
  QCD_CUDA_OK(cudaGetLastError());
  return QCD_OK;
}
