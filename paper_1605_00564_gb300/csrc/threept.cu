// Nucleon three-point functions with the isovector insertions of the axial,
// scalar and tensor charges (Sec. 2.3, eqs. R_A, R_S, R_T), by sequential
// propagators through the sink (fixed sink time t_s):
//
//   C3_Gamma(t) = sum_{x at t_s, y at t} tr[P <N(x) (u-bar Gamma u - d-bar Gamma d)(y) N-bar(x0)>]
//
// Replacing a flavour-f propagator S(x, x0) of the two-point contraction by
// sum_y S(x, y) Gamma S(y, x0) and using S(x, y) = g5 S(y, x)^+ g5:
//
//   Sigma(x) = dC(x)/dS_u(x) - dC(x)/dS_d(x),  C(x) = tr[P G(x)], x at t_s
//   eta      = g5 conj(Sigma)                  (12 sources on the sink time-slice)
//   W        = D^-1 eta                        (12 solves: the sequential propagator)
//   C3(t)    = sum_{y at t} sum_j < W_j(y), g5 Gamma S_j(y) >
//
// with S_j the point-source propagator of source component j and < , > the
// spinor inner product (conjugate-linear in its first argument).  One set of
// 12 solves serves all insertions that share a projector: P+- for the scalar
// density, P53+- = P+- g5 g3 for A_3 = g3 g5 and T_12 = sigma_12.
//
// Normalisation: S and W are solutions of the library's kappa-normalised
// operator; three-point functions of Wilson-normalised propagators are
// (2 kappa)^4 times C3, two-point functions (2 kappa)^3 times C2, so the
// ratios of Sec. 2.3 are R = 2 kappa C3 / C2.
#include <vector>

#include "nucleon_grad.cuh"

qcd_status solver_run(qcd_ctx* c, int n, const double* tol, qcd_rhs_stats* st);

namespace {

using C64 = Cplx<double>;

// 4x4 complex matrices in the chiral basis (row major)
struct Mat4 {
  C64 m[4][4];
};

Mat4 mat_zero() {
  Mat4 o;
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) o.m[i][j] = cmk(0.0, 0.0);
  return o;
}
Mat4 mat_mul(const Mat4& a, const Mat4& b) {
  Mat4 o = mat_zero();
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++)
      for (int k = 0; k < 4; k++) o.m[i][j] = o.m[i][j] + a.m[i][k] * b.m[k][j];
  return o;
}
Mat4 mat_lin(C64 a, const Mat4& x, C64 b, const Mat4& y) {
  Mat4 o;
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) o.m[i][j] = a * x.m[i][j] + b * y.m[i][j];
  return o;
}

// gamma_mu (mu = 0 time) and gamma_5 = diag(1, 1, -1, -1): g0 = [[0, -1], [-1, 0]],
// g_k = [[0, -i s_k], [i s_k, 0]] in 2x2 blocks
Mat4 gamma_matrix(int mu) {
  Mat4 g = mat_zero();
  if (mu == 5) {
    g.m[0][0] = g.m[1][1] = cmk(1.0, 0.0);
    g.m[2][2] = g.m[3][3] = cmk(-1.0, 0.0);
    return g;
  }
  // the 2x2 block e = upper right; lower left = e^+
  C64 e[2][2];
  if (mu == 0) {
    e[0][0] = e[1][1] = cmk(-1.0, 0.0);
    e[0][1] = e[1][0] = cmk(0.0, 0.0);
  } else if (mu == 1) {   // -i s1
    e[0][0] = e[1][1] = cmk(0.0, 0.0);
    e[0][1] = e[1][0] = cmk(0.0, -1.0);
  } else if (mu == 2) {   // -i s2 = [[0, -1], [1, 0]]
    e[0][0] = e[1][1] = cmk(0.0, 0.0);
    e[0][1] = cmk(-1.0, 0.0);
    e[1][0] = cmk(1.0, 0.0);
  } else {                // -i s3 = diag(-i, i)
    e[0][0] = cmk(0.0, -1.0);
    e[1][1] = cmk(0.0, 1.0);
    e[0][1] = e[1][0] = cmk(0.0, 0.0);
  }
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 2; j++) {
      g.m[i][2 + j] = e[i][j];
      g.m[2 + i][j] = conj(e[j][i]);
    }
  return g;
}
Mat4 identity4() {
  Mat4 o = mat_zero();
  for (int i = 0; i < 4; i++) o.m[i][i] = cmk(1.0, 0.0);
  return o;
}

// the projectors and insertions of the three charges
struct ThreePtMats {
  Mat4 P, P53;           // P+- and P53+- = P+- g5 g3
  Mat4 g5G[3];           // g5 Gamma for A_3 = g3 g5, S = 1, T_12 = sigma_12
};
ThreePtMats three_pt_mats(int direction) {
  ThreePtMats o;
  const Mat4 I = identity4(), g0 = gamma_matrix(0), g1 = gamma_matrix(1), g2 = gamma_matrix(2),
             g3 = gamma_matrix(3), g5 = gamma_matrix(5);
  o.P = mat_lin(cmk(0.5, 0.0), I, cmk(direction > 0 ? 0.5 : -0.5, 0.0), g0);
  o.P53 = mat_mul(o.P, mat_mul(g5, g3));
  const Mat4 a3 = mat_mul(g3, g5);
  // sigma_12 = (i/2) [g1, g2]
  const Mat4 s12 = mat_lin(cmk(0.0, 0.5), mat_mul(g1, g2), cmk(0.0, -0.5), mat_mul(g2, g1));
  o.g5G[0] = mat_mul(g5, a3);
  o.g5G[1] = g5;
  o.g5G[2] = mat_mul(g5, s12);
  return o;
}

struct Mats3 {
  double2 m[3][16];
};

// eta = g5 (H_u - H_d): 12 fields, internal FP64 layout
__global__ void k_seq_source(const double2* __restrict__ H, double2* __restrict__ eta, int V) {
  const size_t n = (size_t)12 * 12 * V;
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int comp = (int)((idx / V) % 12);
  const double sg = comp < 6 ? 1.0 : -1.0;     // g5 = diag(1, 1, -1, -1), spin = comp / 3
  const double2 u = H[idx], d = H[n + idx];
  eta[idx] = make_double2(sg * (u.x - d.x), sg * (u.y - d.y));
}

// Per site y: c_k = sum_j < W^{(k)}_j(y), M_k S_j(y) > for the three
// insertions k (M_k = g5 Gamma_k acting on spin, identity on colour), W^{(k)}
// the sequential propagator of the insertion's projector (fields 0..11: P,
// 12..23: P53).  A CTA covers ns sites of one time-slice (rounded up to whole
// warps; the padding threads add zero) and writes its sum to part.
__global__ void k_three_pt(const double2* __restrict__ W, const double2* __restrict__ S, Mats3 mats, int V, int ns,
                           double2* __restrict__ part) {
  const int i = threadIdx.x;
  const int s = blockIdx.x * ns + i;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  if (i < ns) {
    for (int j = 0; j < 12; j++) {
      C64 sv[12];
#pragma unroll
      for (int q = 0; q < 12; q++) {
        const double2 v = S[((size_t)j * 12 + q) * V + s];
        sv[q] = cmk(v.x, v.y);
      }
#pragma unroll
      for (int k = 0; k < 3; k++) {
        const int wset = k == 1 ? 0 : 12;
        C64 sum = cmk(0.0, 0.0);
#pragma unroll
        for (int al = 0; al < 4; al++)
#pragma unroll
          for (int col = 0; col < 3; col++) {
            C64 ms = cmk(0.0, 0.0);
#pragma unroll
            for (int be = 0; be < 4; be++) {
              const double2 m = mats.m[k][4 * al + be];
              ms = ms + cmk(m.x, m.y) * sv[3 * be + col];
            }
            const double2 w = W[((size_t)(wset + j) * 12 + 3 * al + col) * V + s];
            sum = sum + cdot(cmk(w.x, w.y), ms);
          }
        acc[2 * k] += sum.re;
        acc[2 * k + 1] += sum.im;
      }
    }
  }
  __shared__ double red[6][32];
#pragma unroll
  for (int k = 0; k < 6; k++)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0)
    for (int k = 0; k < 6; k++) red[k][w] = acc[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[6] = {0, 0, 0, 0, 0, 0};
    for (int ww = 0; ww < nw; ww++)
      for (int k = 0; k < 6; k++) t[k] += red[k][ww];
    for (int k = 0; k < 3; k++) part[3 * (size_t)blockIdx.x + k] = make_double2(t[2 * k], t[2 * k + 1]);
  }
}

// one thread per (insertion, time-slice): the fixed-order sum of the
// time-slice's partials, re-referenced to the source time
__global__ void k_three_pt_final(const double2* __restrict__ part, int per_t, int T, int t0, double sign,
                                 double2* __restrict__ out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 3 * T) return;
  const int k = idx / T, t = idx % T;
  double2 a = make_double2(0.0, 0.0);
  for (int q = 0; q < per_t; q++) {
    const double2 v = part[3 * ((size_t)t * per_t + q) + k];
    a.x += v.x;
    a.y += v.y;
  }
  out[(size_t)k * T + (t - t0 + T) % T] = make_double2(sign * a.x, sign * a.y);
}

}  // namespace

// Three-point functions of the propagator S_int from the source at src (12
// FP64 fields in the internal layout, not in wsD[0..3] or wsD[5..7]), sink
// at src_t + direction t_sep.  S_sink is the same propagator as seen at the
// sink (S_int itself for a point sink; K S_int with the Gaussian kernel K of
// a smeared sink, in which case the sequential source is smeared with K as
// well, K being Hermitian).  Sequential solves to tol, or with n_iter > 0
// exactly n_iter GCR iterations each (the fixed-iteration sloppy mode of
// Sec. 3, Table 3; such solves count as successful).  corr3: host [3][T][2];
// st: 24 entries.
qcd_status threept_internal(qcd_ctx* c, const void* S_int, const void* S_sink, const int src[4], int t_sep,
                            int direction, double tol, int n_iter, double* corr3, qcd_rhs_stats* st) {
  const int V = c->g.V, T = c->g.L[0], L3 = V / T;
  const int t0 = src[0];
  const int ts = ((t0 + direction * t_sep) % T + T) % T;
  const int bc3 = c->g.bc_t * c->g.bc_t * c->g.bc_t;
  const double sign = ts < t0 ? (double)bc3 : 1.0;   // as the two-point function's wrapped sink times
  const size_t f64 = spinor_bytes(c, QCD_PREC_F64);
  // H (24: u, d) in wsD[5]; eta (24: P, P53) in wsD[6]; W (24) in wsD[7]
  QCD_TRY(devbuf_ensure(c->wsD[5], f64 * 24));
  QCD_TRY(devbuf_ensure(c->wsD[6], f64 * 24));
  QCD_TRY(devbuf_ensure(c->wsD[7], f64 * 24));
  const ThreePtMats M = three_pt_mats(direction);
  int ns = 8;
  while (L3 % ns) ns >>= 1;
  const size_t smem = sizeof(C64) * 144 * ns;
  QCD_CUDA_OK(cudaFuncSetAttribute(nucleon_grad::k_dC_dS, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  std::vector<double2> pm(16 * (size_t)T);
  for (int p = 0; p < 2; p++) {
    const Mat4& P = p == 0 ? M.P : M.P53;
    for (auto& v : pm) v = make_double2(0.0, 0.0);
    for (int i = 0; i < 4; i++)
      for (int j = 0; j < 4; j++) pm[16 * (size_t)ts + 4 * i + j] = make_double2(P.m[i][j].re, P.m[i][j].im);
    QCD_TRY(devbuf_ensure(c->contract, sizeof(double2) * 16 * T));
    QCD_CUDA_OK(cudaMemcpyAsync(c->contract.p, pm.data(), sizeof(double2) * 16 * T, cudaMemcpyHostToDevice,
                                c->stream));
    QCD_CUDA_OK(cudaMemsetAsync(c->wsD[5].p, 0, f64 * 24, c->stream));
    {
      // the sequential source lives on the sink time-slice only
      ProfScope ps(c, FAM_CONTRACT, (double)L3 * 3 * 2304, (double)L3 * 36 * 6 * 200 * 8);
      nucleon_grad::k_dC_dS<<<L3 / ns, 18 * ns, smem, c->stream>>>((const double2*)S_sink,
                                                                  (const double2*)c->contract.p, V, L3, ns, ts * L3,
                                                                  (double2*)c->wsD[5].p);
      QCD_CUDA_OK(cudaGetLastError());
      const size_t n = (size_t)144 * V;
      k_seq_source<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(
          (const double2*)c->wsD[5].p, (double2*)((char*)c->wsD[6].p + f64 * 12 * p), V);
      QCD_CUDA_OK(cudaGetLastError());
    }
    if (S_sink != S_int) QCD_TRY(smear_fields(c, (char*)c->wsD[6].p + f64 * 12 * p, 12));
  }
  // the 24 sequential propagators, 12 at a time: W = D^-1 eta
  std::vector<double> tols(12, n_iter > 0 ? 1e-300 : tol);
  const int max_outer = c->params.max_outer;
  if (n_iter > 0) c->params.max_outer = n_iter;
  qcd_status rc = QCD_OK;
  for (int p = 0; p < 2 && rc == QCD_OK; p++) {
    if ((rc = devbuf_ensure(c->wsD[0], f64 * 12)) != QCD_OK) break;
    if ((rc = devbuf_ensure(c->wsD[1], f64 * 12)) != QCD_OK) break;
    if (cudaMemcpyAsync(c->wsD[0].p, (char*)c->wsD[6].p + f64 * 12 * p, f64 * 12, cudaMemcpyDeviceToDevice,
                        c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->wsD[1].p, 0, f64 * 12, c->stream) != cudaSuccess) {
      qcd_set_error("sequential source set-up failed");
      rc = QCD_ERR_CUDA;
      break;
    }
    if ((rc = solver_run(c, 12, tols.data(), st + 12 * p)) != QCD_OK) break;
    if (cudaMemcpyAsync((char*)c->wsD[7].p + f64 * 12 * p, c->wsD[1].p, f64 * 12, cudaMemcpyDeviceToDevice,
                        c->stream) != cudaSuccess) {
      qcd_set_error("sequential propagator copy failed");
      rc = QCD_ERR_CUDA;
    }
  }
  c->params.max_outer = max_outer;
  QCD_TRY(rc);
  if (n_iter > 0)
    for (int r = 0; r < 24; r++)
      if (st[r].status == QCD_ERR_NOT_CONVERGED) st[r].status = QCD_OK;   // stopped at n_iter by design
  // contraction with the forward propagator, per time-slice
  int cs = 128;
  while (L3 % cs) cs >>= 1;
  const int nb = V / cs, per_t = L3 / cs;
  QCD_TRY(devbuf_ensure(c->contract, sizeof(double2) * (3 * (size_t)nb + 3 * T)));
  double2* part = (double2*)c->contract.p;
  double2* cd = part + 3 * (size_t)nb;
  Mats3 mats;
  for (int k = 0; k < 3; k++)
    for (int i = 0; i < 4; i++)
      for (int j = 0; j < 4; j++) mats.m[k][4 * i + j] = make_double2(M.g5G[k].m[i][j].re, M.g5G[k].m[i][j].im);
  {
    ProfScope ps(c, FAM_CONTRACT, (double)V * 36 * 192, (double)V * 12 * 3 * 12 * (4 * 8 + 8));
    const int threads = cs < 32 ? 32 : cs;
    k_three_pt<<<nb, threads, 0, c->stream>>>((const double2*)c->wsD[7].p, (const double2*)S_int, mats, V, cs,
                                              part);
    QCD_CUDA_OK(cudaGetLastError());
    k_three_pt_final<<<(3 * T + 127) / 128, 128, 0, c->stream>>>(part, per_t, T, t0, sign, cd);
    QCD_CUDA_OK(cudaGetLastError());
  }
  QCD_CUDA_OK(cudaMemcpyAsync(corr3, cd, sizeof(double2) * 3 * T, cudaMemcpyDeviceToHost, c->stream));
  QCD_CUDA_OK(cudaStreamSynchronize(c->stream));
  return QCD_OK;
}

extern "C" qcd_status qcd_nucleon_3pt(qcd_ctx* c, const double* prop, const int src[4], int t_sep, int direction,
                                      double tol, double* corr3, qcd_rhs_stats* stats) {
  if (!c || !prop || !src || !corr3) {
    qcd_set_error("null argument");
    return QCD_ERR_ARG;
  }
  if (!c->have_gauge) {
    qcd_set_error("no gauge field loaded");
    return QCD_ERR_STATE;
  }
  const int T = c->g.L[0];
  for (int mu = 0; mu < 4; mu++)
    if (src[mu] < 0 || src[mu] >= c->g.L[mu]) {
      qcd_set_error("source outside the lattice");
      return QCD_ERR_ARG;
    }
  if (t_sep < 1 || t_sep >= T) {
    qcd_set_error("t_sep must be in [1, T)");
    return QCD_ERR_ARG;
  }
  if (direction != 1 && direction != -1) {
    qcd_set_error("direction must be +1 (forward, P+) or -1 (backward, P-)");
    return QCD_ERR_ARG;
  }
  if (!(tol > 0 && tol < 1)) {
    qcd_set_error("tol must be in (0, 1)");
    return QCD_ERR_ARG;
  }
  const size_t f64 = spinor_bytes(c, QCD_PREC_F64);
  QCD_TRY(devbuf_ensure(c->wsD[4], f64 * 12));
  QCD_TRY(layout_spinor_import(c, prop, c->wsD[4].p, QCD_PREC_F64, 12));
  std::vector<qcd_rhs_stats> st(24);
  QCD_TRY(threept_internal(c, c->wsD[4].p, c->wsD[4].p, src, t_sep, direction, tol, 0, corr3, st.data()));
  qcd_status worst = QCD_OK;
  for (int r = 0; r < 24; r++) {
    if (stats) stats[r] = st[r];
    if (st[r].status != QCD_OK && worst == QCD_OK) worst = (qcd_status)st[r].status;
  }
  return worst;
}
