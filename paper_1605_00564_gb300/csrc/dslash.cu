// The Wilson-clover operator D (Sec. 2.2, the Dirac equation D psi = eta):
//   D psi(x) = A(x) psi(x) - kappa sum_mu [(1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^+ psi(x-mu)]
// with A(x) = 1 + clover term; D^+ exchanges the two spin projectors.
//
// One thread per (site, right-hand side).  The CTAs of all right-hand sides
// that cover the same run of sites are adjacent in launch order, so the
// gauge and clover words of those sites are reused from L2 across the RHS.
// Every (1 -+ g_mu) projection halves the spinor before the SU(3) multiply.
#include "qcd_internal.cuh"

namespace {

constexpr int DSLASH_TPB = 128;

template <typename F, int MU, int DAGGER>
__device__ inline void hop_dir(Spinor<typename F::R>& acc, const void* in, const void* gauge, const Geom& g, int s,
                               const int c[4], typename F::R scale) {
  using R = typename F::R;
  constexpr int SF = DAGGER ? +1 : -1;   // projector sign for the forward hop
  constexpr int SB = -SF;                // and for the backward hop
  const int V = g.V;
  // acc += scale * (1 SF g_mu) U_mu(x) psi(x + mu)
  {
    int sf = site_fwd(g, s, c, MU);
    R sign = (MU == 0 && c[0] == g.L[0] - 1) ? (R)g.bc_t * scale : scale;
    HalfSpinor<R> h = project<MU, SF>(F::load_spinor(in, V, sf));
    h = su3_mul(F::load_link(gauge, V, MU, s), h);
    accum_recon<MU, SF>(acc, h, sign);
  }
  // acc += scale * (1 SB g_mu) U_mu(x - mu)^+ psi(x - mu)
  {
    int sb = site_bwd(g, s, c, MU);
    R sign = (MU == 0 && c[0] == 0) ? (R)g.bc_t * scale : scale;
    HalfSpinor<R> h = project<MU, SB>(F::load_spinor(in, V, sb));
    h = su3_dag_mul(F::load_link(gauge, V, MU, sb), h);
    accum_recon<MU, SB>(acc, h, sign);
  }
}

// O: storage of the output (F itself, or FieldsH for FP16 + per-site scale)
template <typename F, typename O, int DAGGER>
__global__ void __launch_bounds__(DSLASH_TPB) k_dslash(const char* __restrict__ in, char* __restrict__ out,
                                                       const void* __restrict__ gauge, const void* __restrict__ clover,
                                                       Geom g, typename F::R kappa, int nrhs, const int* mask) {
  using R = typename F::R;
  const int rhs = blockIdx.x % nrhs;
  const int s = (blockIdx.x / nrhs) * DSLASH_TPB + threadIdx.x;
  if (s >= g.V) return;
  if (mask && !mask[rhs]) return;
  const size_t off = (size_t)rhs * F::spinor_bytes * g.V;
  const size_t off_out = (size_t)rhs * O::spinor_bytes * g.V;
  const void* src = in + off;
  int c[4];
  site_coords(g, s, c);
  Spinor<R> o = clover_apply<F>(clover, g.V, s, F::load_spinor(src, g.V, s));
  hop_dir<F, 0, DAGGER>(o, src, gauge, g, s, c, -kappa);
  hop_dir<F, 1, DAGGER>(o, src, gauge, g, s, c, -kappa);
  hop_dir<F, 2, DAGGER>(o, src, gauge, g, s, c, -kappa);
  hop_dir<F, 3, DAGGER>(o, src, gauge, g, s, c, -kappa);
  O::store_spinor(out + off_out, g.V, s, o);
}

template <typename F, typename O = F>
qcd_status launch(qcd_ctx* c, const void* in, void* out, const void* gauge, const void* clover, int nrhs, int dagger,
                  const int* mask) {
  int nb = (c->g.V + DSLASH_TPB - 1) / DSLASH_TPB;
  dim3 grid((unsigned)nb * nrhs);
  if (dagger)
    k_dslash<F, O, 1><<<grid, DSLASH_TPB, 0, c->stream>>>((const char*)in, (char*)out, gauge, clover, c->g,
                                                          (typename F::R)c->kappa, nrhs, mask);
  else
    k_dslash<F, O, 0><<<grid, DSLASH_TPB, 0, c->stream>>>((const char*)in, (char*)out, gauge, clover, c->g,
                                                          (typename F::R)c->kappa, nrhs, mask);
  QCD_CUDA_OK(cudaGetLastError());
  return QCD_OK;
}

}  // namespace

// Algorithmic cost per site: each input spinor read once, the output written
// once, the 4 links of the site and its clover term read once per launch;
// 1320 flops for the eight spin-projected hops and 504 for the clover term.
// out_prec = QCD_PREC_H16 (FP32 input only): the output is stored as FP16 with
// a per-site scale.
qcd_status dslash_apply(qcd_ctx* c, const void* in, void* out, int prec, int nrhs, int dagger, const int* mask,
                        int nactive, int out_prec) {
  const double V = c->g.V;
  if (prec == QCD_PREC_F64) {
    ProfScope ps(c, FAM_DSLASH_D, V * (nactive * 2.0 * 192 + 4 * 144 + 576), V * nactive * 1824.0);
    return launch<FieldsD>(c, in, out, c->gaugeD.p, c->cloverD.p, nrhs, dagger, mask);
  }
  if (out_prec == QCD_PREC_H16) {
    ProfScope ps(c, FAM_DSLASH_F, V * (nactive * (96.0 + FieldsH::spinor_bytes) + 4 * 48 + 288), V * nactive * 1824.0);
    return launch<FieldsF, FieldsH>(c, in, out, c->gaugeF.p, c->cloverF.p, nrhs, dagger, mask);
  }
  ProfScope ps(c, FAM_DSLASH_F, V * (nactive * 2.0 * 96 + 4 * 48 + 288), V * nactive * 1824.0);
  return launch<FieldsF>(c, in, out, c->gaugeF.p, c->cloverF.p, nrhs, dagger, mask);
}
