// The Wilson-clover operator D (Sec. 2.2, the Dirac equation D psi = eta):
//   D psi(x) = A(x) psi(x) - kappa sum_mu [(1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^+ psi(x-mu)]
// with A(x) = 1 + clover term; D^+ exchanges the two spin projectors.
//
// One thread per (site, right-hand side).  The CTAs of all right-hand sides
// that cover the same run of sites are adjacent in launch order, so the
// gauge and clover words of those sites are reused from L2 across the RHS.
// Every (1 -+ g_mu) projection halves the spinor before the SU(3) multiply.
//
// Traversal order with several RHS: a run of DSLASH_TPB sites is part of one
// (t, z) plane; runs are visited slab by slab, a slab being zw consecutive z
// planes, and within a slab time-slice by time-slice.  A site's neighbours in
// t are then zw planes (zw X Y sites) away in launch order instead of a whole
// time-slice: with 12 RHS a time-slice of 32^3 sites moves ~75 MB, more than
// L2 keeps, while a slab of 8 planes moves ~20 MB, so the t-neighbours'
// spinors are still in L2 when they are read.
#include "qcd_internal.cuh"

namespace {

constexpr int DSLASH_TPB = 128;

// cp: runs of DSLASH_TPB sites per (t, z) plane (0: plain lexicographic
// order); zw: z planes per slab
struct RunOrder {
  int cp, zw;
};

// first site of run q
__device__ inline int run_base(const Geom& g, RunOrder o, int q) {
  if (o.cp == 0) return q * DSLASH_TPB;
  const int per_t = o.zw * o.cp;
  const int per_slab = g.L[0] * per_t;
  const int zb = q / per_slab;
  int r = q - zb * per_slab;
  const int t = r / per_t;
  r -= t * per_t;
  const int z = zb * o.zw + r / o.cp;
  const int run = r % o.cp;
  return (t * g.L[3] + z) * g.L[2] * g.L[1] + run * DSLASH_TPB;
}

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
                                                       Geom g, typename F::R kappa, int nrhs, const int* mask,
                                                       RunOrder ord) {
  using R = typename F::R;
  const int rhs = blockIdx.x % nrhs;
  const int s = run_base(g, ord, blockIdx.x / nrhs) + threadIdx.x;
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
  // slab order with several RHS when a (t, z) plane holds whole runs
  RunOrder ord = {0, 1};
  const int plane = c->g.L[1] * c->g.L[2];
  if (nrhs > 1 && plane % DSLASH_TPB == 0) {
    ord.cp = plane / DSLASH_TPB;
    ord.zw = c->g.L[3] % 8 == 0 ? 8 : c->g.L[3] % 4 == 0 ? 4 : c->g.L[3] % 2 == 0 ? 2 : 1;
  }
  if (dagger)
    k_dslash<F, O, 1><<<grid, DSLASH_TPB, 0, c->stream>>>((const char*)in, (char*)out, gauge, clover, c->g,
                                                          (typename F::R)c->kappa, nrhs, mask, ord);
  else
    k_dslash<F, O, 0><<<grid, DSLASH_TPB, 0, c->stream>>>((const char*)in, (char*)out, gauge, clover, c->g,
                                                          (typename F::R)c->kappa, nrhs, mask, ord);
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
