// Smeared sources and sinks (Sec. 2.3: Gaussian smearing at source and sink
// with APE-smeared gauge links in the Laplacian).  The paper takes method and
// parameters by citation; the readings implemented here:
//
// APE smearing of the spatial links k = 1, 2, 3, one step:
//   V_k(x) = U_k(x) + alpha sum_{j spatial, j != k} [ U_j(x) U_k(x+j) U_j(x+k)^+
//                                                   + U_j(x-j)^+ U_k(x-j) U_j(x-j+k) ]
//   U'_k(x) = W det(W)^(-1/3),  W the unitary factor of the polar
//             decomposition V = W (V^+ V)^(1/2), principal cube root;
// time links are copied unchanged.  W is computed by Newton's iteration for
// the polar decomposition (Higham 1986): W <- (W + W^-+) / 2 from V scaled to
// unit root-mean-square singular value, a fixed number of steps.
//
// Gaussian smearing, one step (spin untouched, periodic in space):
//   psi'(x) = [psi(x) + kappa_G sum_k (U_k(x) psi(x+k) + U_k(x-k)^+ psi(x-k))] / (1 + 6 kappa_G),
// applied n times with the APE-smeared links.  The kernel is Hermitian, so a
// smeared sink is the same operator on the sink index of a propagator.
#include <math.h>

#include "qcd_internal.cuh"

namespace {

using C64 = Cplx<double>;
struct M3 {
  C64 m[3][3];
};

constexpr int kNewtonSteps = 20;

__device__ inline M3 m3_mul(const M3& a, const M3& b) {
  M3 o;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      C64 s = a.m[i][0] * b.m[0][j];
      cmac(s, a.m[i][1], b.m[1][j]);
      cmac(s, a.m[i][2], b.m[2][j]);
      o.m[i][j] = s;
    }
  return o;
}
// a b^+
__device__ inline M3 m3_mul_dag(const M3& a, const M3& b) {
  M3 o;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      C64 s = a.m[i][0] * conj(b.m[j][0]);
      cmac(s, a.m[i][1], conj(b.m[j][1]));
      cmac(s, a.m[i][2], conj(b.m[j][2]));
      o.m[i][j] = s;
    }
  return o;
}
// a^+ b
__device__ inline M3 m3_dag_mul(const M3& a, const M3& b) {
  M3 o;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      C64 s = conj(a.m[0][i]) * b.m[0][j];
      cmac(s, conj(a.m[1][i]), b.m[1][j]);
      cmac(s, conj(a.m[2][i]), b.m[2][j]);
      o.m[i][j] = s;
    }
  return o;
}

__device__ inline M3 load_m3(const double2* U, int V, int mu, int s) {
  M3 o;
#pragma unroll
  for (int k = 0; k < 9; k++) {
    const double2 v = U[((size_t)mu * 9 + k) * V + s];
    o.m[k / 3][k % 3] = cmk(v.x, v.y);
  }
  return o;
}
__device__ inline void store_m3(double2* U, int V, int mu, int s, const M3& a) {
#pragma unroll
  for (int k = 0; k < 9; k++) U[((size_t)mu * 9 + k) * V + s] = make_double2(a.m[k / 3][k % 3].re, a.m[k / 3][k % 3].im);
}

// the projection onto SU(3) described above
__device__ inline M3 project_su3(M3 W) {
  double f = 0;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) f += W.m[i][j].re * W.m[i][j].re + W.m[i][j].im * W.m[i][j].im;
  const double sc = f > 0 ? sqrt(3.0 / f) : 1.0;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) W.m[i][j] = sc * W.m[i][j];
  for (int it = 0; it < kNewtonSteps; it++) {
    // (W^-1)^+ = conj(cofactor(W)) / conj(det W)
    M3 cof;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
      for (int j = 0; j < 3; j++) {
        const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
        cof.m[i][j] = W.m[i1][j1] * W.m[i2][j2] - W.m[i1][j2] * W.m[i2][j1];
      }
    const C64 det = W.m[0][0] * cof.m[0][0] + W.m[0][1] * cof.m[0][1] + W.m[0][2] * cof.m[0][2];
    const double dn = det.re * det.re + det.im * det.im;
    // 1 / conj(det) = det / |det|^2
    const C64 idc = cmk(det.re / dn, det.im / dn);
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
      for (int j = 0; j < 3; j++) W.m[i][j] = 0.5 * (W.m[i][j] + conj(cof.m[i][j]) * idc);
  }
  // divide out the determinant's phase (principal cube root)
  C64 cof0 = W.m[1][1] * W.m[2][2] - W.m[1][2] * W.m[2][1];
  C64 cof1 = W.m[1][2] * W.m[2][0] - W.m[1][0] * W.m[2][2];
  C64 cof2 = W.m[1][0] * W.m[2][1] - W.m[1][1] * W.m[2][0];
  const C64 det = W.m[0][0] * cof0 + W.m[0][1] * cof1 + W.m[0][2] * cof2;
  const double ph = -atan2(det.im, det.re) / 3.0;
  const C64 z = cmk(cos(ph), sin(ph));
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) W.m[i][j] = z * W.m[i][j];
  return W;
}

// one APE step: Uout = smeared spatial links of Uin, time links copied
__global__ void k_ape_step(const double2* __restrict__ Uin, double2* __restrict__ Uout, Geom g, double alpha) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int c[4];
  site_coords(g, s, c);
  store_m3(Uout, g.V, 0, s, load_m3(Uin, g.V, 0, s));
  for (int k = 1; k < 4; k++) {
    M3 V = load_m3(Uin, g.V, k, s);
    const int sk = site_fwd(g, s, c, k);
    for (int j = 1; j < 4; j++) {
      if (j == k) continue;
      const int sj = site_fwd(g, s, c, j);
      const int smj = site_bwd(g, s, c, j);
      int cmj[4] = {c[0], c[1], c[2], c[3]};
      cmj[j] = (c[j] + g.L[j] - 1) % g.L[j];
      const int smjk = site_fwd(g, smj, cmj, k);
      // U_j(x) U_k(x+j) U_j(x+k)^+
      const M3 f = m3_mul_dag(m3_mul(load_m3(Uin, g.V, j, s), load_m3(Uin, g.V, k, sj)), load_m3(Uin, g.V, j, sk));
      // U_j(x-j)^+ U_k(x-j) U_j(x-j+k)
      const M3 b = m3_mul(m3_dag_mul(load_m3(Uin, g.V, j, smj), load_m3(Uin, g.V, k, smj)), load_m3(Uin, g.V, j, smjk));
#pragma unroll
      for (int p = 0; p < 3; p++)
#pragma unroll
        for (int q = 0; q < 3; q++) V.m[p][q] = V.m[p][q] + alpha * (f.m[p][q] + b.m[p][q]);
    }
    store_m3(Uout, g.V, k, s, project_su3(V));
  }
}

// one Gaussian step on nrhs FP64 internal spinors
__global__ void k_gauss_step(const double2* __restrict__ in, double2* __restrict__ out, const double2* __restrict__ U,
                             Geom g, double kappa, int nrhs) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)g.V * nrhs) return;
  const int s = (int)(idx % g.V);
  const size_t r = idx / g.V;
  const double2* p = in + r * 12 * (size_t)g.V;
  int c[4];
  site_coords(g, s, c);
  C64 acc[12];
#pragma unroll
  for (int q = 0; q < 12; q++) {
    const double2 v = p[(size_t)q * g.V + s];
    acc[q] = cmk(v.x, v.y);
  }
  for (int k = 1; k < 4; k++) {
    const int sf = site_fwd(g, s, c, k), sb = site_bwd(g, s, c, k);
    const M3 Uf = load_m3(U, g.V, k, s), Ub = load_m3(U, g.V, k, sb);
#pragma unroll
    for (int sp = 0; sp < 4; sp++)
#pragma unroll
      for (int a = 0; a < 3; a++) {
        C64 h = cmk(0.0, 0.0);
#pragma unroll
        for (int b = 0; b < 3; b++) {
          const double2 vf = p[(size_t)(3 * sp + b) * g.V + sf], vb = p[(size_t)(3 * sp + b) * g.V + sb];
          cmac(h, Uf.m[a][b], cmk(vf.x, vf.y));
          cmac_conj(h, Ub.m[b][a], cmk(vb.x, vb.y));
        }
        acc[3 * sp + a] = acc[3 * sp + a] + kappa * h;
      }
  }
  const double nrm = 1.0 / (1.0 + 6.0 * kappa);
  double2* o = out + r * 12 * (size_t)g.V;
#pragma unroll
  for (int q = 0; q < 12; q++) o[(size_t)q * g.V + s] = make_double2(nrm * acc[q].re, nrm * acc[q].im);
}

// internal FP64 gauge [4][9][V] -> canonical [site][mu][3][3]
__global__ void k_gauge_export(const double2* __restrict__ U, double2* __restrict__ out, int V) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)V * 36) return;
  const int s = (int)(idx / 36), e = (int)(idx % 36);
  out[idx] = U[(size_t)e * V + s];
}

}  // namespace

qcd_status smear_fields(qcd_ctx* c, void* fields, int nrhs) {
  if (c->smear_n == 0) return QCD_OK;
  const size_t bytes = spinor_bytes(c, QCD_PREC_F64) * nrhs;
  QCD_TRY(devbuf_ensure(c->smearbuf[0], bytes));
  const size_t n = (size_t)c->g.V * nrhs;
  ProfScope ps(c, FAM_LAYOUT, (double)n * c->smear_n * 2 * 192, (double)n * c->smear_n * 3 * 2 * 4 * 3 * 8 * 3);
  void* a = fields;
  void* b = c->smearbuf[0].p;
  for (int it = 0; it < c->smear_n; it++) {
    k_gauss_step<<<(unsigned)((n + 127) / 128), 128, 0, c->stream>>>((const double2*)a, (double2*)b,
                                                                     (const double2*)c->gaugeS.p, c->g, c->smear_kappa,
                                                                     nrhs);
    QCD_CUDA_OK(cudaGetLastError());
    void* t = a;
    a = b;
    b = t;
  }
  if (a != fields) QCD_CUDA_OK(cudaMemcpyAsync(fields, a, bytes, cudaMemcpyDeviceToDevice, c->stream));
  return QCD_OK;
}

extern "C" qcd_status qcd_smear_links(qcd_ctx* c, double alpha, int n_ape) {
  if (!c) {
    qcd_set_error("null context");
    return QCD_ERR_ARG;
  }
  if (!c->have_gauge) {
    qcd_set_error("no gauge field loaded");
    return QCD_ERR_STATE;
  }
  if (!(isfinite(alpha) && alpha >= 0) || n_ape < 0 || n_ape > 1000) {
    qcd_set_error("need alpha >= 0 and 0 <= n_ape <= 1000");
    return QCD_ERR_ARG;
  }
  const size_t bytes = (size_t)c->g.V * 36 * sizeof(double2);
  QCD_TRY(devbuf_ensure(c->gaugeS, bytes));
  QCD_CUDA_OK(cudaMemcpyAsync(c->gaugeS.p, c->gaugeD.p, bytes, cudaMemcpyDeviceToDevice, c->stream));
  if (n_ape > 0) {
    DevBuf tmp;
    QCD_TRY(devbuf_ensure(tmp, bytes));
    void* a = c->gaugeS.p;
    void* b = tmp.p;
    for (int it = 0; it < n_ape; it++) {
      k_ape_step<<<(c->g.V + 127) / 128, 128, 0, c->stream>>>((const double2*)a, (double2*)b, c->g, alpha);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) {
        devbuf_free(tmp);
        qcd_set_error("APE step: %s", cudaGetErrorString(e));
        return QCD_ERR_CUDA;
      }
      void* t = a;
      a = b;
      b = t;
    }
    cudaError_t e = a != c->gaugeS.p ? cudaMemcpyAsync(c->gaugeS.p, a, bytes, cudaMemcpyDeviceToDevice, c->stream)
                                     : cudaSuccess;
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    devbuf_free(tmp);
    if (e != cudaSuccess) {
      qcd_set_error("APE smearing: %s", cudaGetErrorString(e));
      return QCD_ERR_CUDA;
    }
  }
  QCD_CUDA_OK(cudaStreamSynchronize(c->stream));
  c->have_smeared_links = 1;
  return QCD_OK;
}

extern "C" qcd_status qcd_set_smearing(qcd_ctx* c, double kappa_g, int n_gauss) {
  if (!c) {
    qcd_set_error("null context");
    return QCD_ERR_ARG;
  }
  if (!(isfinite(kappa_g) && kappa_g >= 0) || n_gauss < 0 || n_gauss > 10000) {
    qcd_set_error("need kappa_g >= 0 and 0 <= n_gauss <= 10000");
    return QCD_ERR_ARG;
  }
  if (n_gauss > 0 && !c->have_smeared_links) {
    qcd_set_error("qcd_smear_links must come first");
    return QCD_ERR_STATE;
  }
  c->smear_kappa = kappa_g;
  c->smear_n = n_gauss;
  return QCD_OK;
}

extern "C" qcd_status qcd_smear_gaussian(qcd_ctx* c, const double* in, double* out, int nrhs) {
  if (!c || !in || !out || nrhs < 1) {
    qcd_set_error("bad argument");
    return QCD_ERR_ARG;
  }
  if (!c->have_smeared_links) {
    qcd_set_error("qcd_smear_links must come first");
    return QCD_ERR_STATE;
  }
  const size_t b = spinor_bytes(c, QCD_PREC_F64) * nrhs;
  QCD_TRY(devbuf_ensure(c->smearbuf[1], b));
  QCD_TRY(layout_spinor_import(c, in, c->smearbuf[1].p, QCD_PREC_F64, nrhs));
  QCD_TRY(smear_fields(c, c->smearbuf[1].p, nrhs));
  QCD_TRY(layout_spinor_export(c, c->smearbuf[1].p, out, QCD_PREC_F64, nrhs));
  QCD_CUDA_OK(cudaStreamSynchronize(c->stream));
  return QCD_OK;
}

extern "C" qcd_status qcd_get_smeared_links(qcd_ctx* c, double* out) {
  if (!c || !out) {
    qcd_set_error("bad argument");
    return QCD_ERR_ARG;
  }
  if (!c->have_smeared_links) {
    qcd_set_error("qcd_smear_links must come first");
    return QCD_ERR_STATE;
  }
  const size_t n = (size_t)c->g.V * 36;
  k_gauge_export<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>((const double2*)c->gaugeS.p, (double2*)out,
                                                                     c->g.V);
  QCD_CUDA_OK(cudaGetLastError());
  QCD_CUDA_OK(cudaStreamSynchronize(c->stream));
  return QCD_OK;
}
