// qcd_nucleon_2pt_noalloc: the nucleon two-point contraction without any
// device allocation.
//
// Who needs it: callers that cannot call cudaMalloc at the point where they
// want the correlator.  A stream being captured into a CUDA graph cannot
// record an allocation; a host application whose device memory is owned by
// another allocator (a framework's caching pool, a fixed arena set up at start)
// must not have a library grab memory behind its back; and a latency-critical
// loop cannot afford an allocation's implicit synchronisation.  These callers
// bring every buffer themselves.  This entry point needs no context and no
// workspace: its only scratch, the per-CTA partial sums of the contraction,
// lives in a file-scope __device__ array of fixed size that every GPU loading
// the library holds until the process exits.
//
// The contraction is the same as qcd_nucleon_2pt's (the Wick contractions of
// N = eps^{abc} (u^a^T C g5 d^b) u^c with u = d, projected with
// P+- = (1 +- g0)/2 and summed over each timeslice), but the kernel reads the
// propagator directly in the canonical layout [rhs][site][spin][colour] and
// writes the correlator to device memory.
#include <mutex>

#include "qcd_internal.cuh"

// Largest number of partial sums held in the static scratch: two (P+ and P-)
// per CTA of 32 sites, i.e. V <= 32 * 131072 = 4,194,304 sites (e.g. 32^3 x 128
// or 40^3 x 64).  4 MiB of device memory.
#define QCD_NOALLOC_MAX_CTAS 131072

static __device__ __align__(256) double2 g_nucleon_scratch[2 * QCD_NOALLOC_MAX_CTAS];

namespace {

__constant__ int c_perm_na[6][4] = {  // a, b, c, sign
    {0, 1, 2, 1}, {1, 2, 0, 1}, {2, 0, 1, 1}, {0, 2, 1, -1}, {2, 1, 0, -1}, {1, 0, 2, -1}};

template <typename R>
__device__ inline Cplx<R> Sat(const Cplx<R>* S_s, int ns, int i, int al, int a, int alp, int ap) {
  return S_s[((3 * al + a) * 12 + 3 * alp + ap) * ns + i];
}
template <typename R>
__device__ inline R gsg(int b) { return (b & 1) ? (R)1 : (R)-1; }

// prop canonical: entry (rhs, site, comp) at prop[(rhs * V + site) * 12 + comp]
template <typename R>
__global__ void k_nucleon_canonical(const double2* __restrict__ prop, int V, int ns, double2* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cplx<R>* S_s = (Cplx<R>*)smem_raw;
  const int s0 = blockIdx.x * ns;
  for (int idx = threadIdx.x; idx < 144 * ns; idx += blockDim.x) {
    int i = idx % ns, e = idx / ns;
    int comp = e / 12, rhs = e - comp * 12;
    double2 v = prop[((size_t)rhs * V + s0 + i) * 12 + comp];
    S_s[e * ns + i] = cmk((R)v.x, (R)v.y);
  }
  __syncthreads();
  const int i = threadIdx.x % ns;
  const int pq = threadIdx.x / ns;
  const int a = c_perm_na[pq][0], b = c_perm_na[pq][1], c = c_perm_na[pq][2];
  const R eps = (R)c_perm_na[pq][3];
  Cplx<R> accp = cmk((R)0, (R)0), accm = cmk((R)0, (R)0);
#pragma unroll 1
  for (int q = 0; q < 6; q++) {
    const int ap = c_perm_na[q][0], bp = c_perm_na[q][1], cp = c_perm_na[q][2];
    const R ee = eps * (R)c_perm_na[q][3];
    Cplx<R> T = cmk((R)0, (R)0);
#pragma unroll
    for (int be = 0; be < 4; be++)
#pragma unroll
      for (int bq = 0; bq < 4; bq++)
        T = T + (gsg<R>(be) * gsg<R>(bq)) * (Sat(S_s, ns, i, be, a, bq, ap) * Sat(S_s, ns, i, be ^ 1, b, bq ^ 1, bp));
    Cplx<R> d = cmk((R)0, (R)0), o = cmk((R)0, (R)0);
#pragma unroll
    for (int l = 0; l < 4; l++) {
      d = d + Sat(S_s, ns, i, l, c, l, cp);
      o = o + Sat(S_s, ns, i, l ^ 2, c, l, cp);
    }
    Cplx<R> t1p = T * ((R)0.5 * (d - o)), t1m = T * ((R)0.5 * (d + o));
    Cplx<R> Y[4][4];
#pragma unroll
    for (int ii = 0; ii < 4; ii++)
#pragma unroll
      for (int j = 0; j < 4; j++) {
        Cplx<R> y = cmk((R)0, (R)0);
#pragma unroll
        for (int k = 0; k < 4; k++)
          y = y + (gsg<R>(k) * gsg<R>(j)) * (Sat(S_s, ns, i, ii, c, k, ap) * Sat(S_s, ns, i, j ^ 1, b, k ^ 1, bp));
        Y[ii][j] = y;
      }
    Cplx<R> zd = cmk((R)0, (R)0), zo = cmk((R)0, (R)0);
#pragma unroll
    for (int l = 0; l < 4; l++)
#pragma unroll
      for (int k = 0; k < 4; k++) {
        Cplx<R> sv = Sat(S_s, ns, i, k, a, l, cp);
        zd = zd + Y[l][k] * sv;
        zo = zo + Y[l ^ 2][k] * sv;
      }
    accp = accp + ee * (t1p - (R)0.5 * (zd - zo));
    accm = accm + ee * (t1m - (R)0.5 * (zd + zo));
  }
  __shared__ double red[4][32];
  double v[4] = {(double)accp.re, (double)accp.im, (double)accm.re, (double)accm.im};
#pragma unroll
  for (int k = 0; k < 4; k++)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  if (lane == 0)
    for (int k = 0; k < 4; k++) red[k][w] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[4] = {0, 0, 0, 0};
    for (int ww = 0; ww < nw; ww++)
      for (int k = 0; k < 4; k++) t[k] += red[k][ww];
    part[2 * (size_t)blockIdx.x] = make_double2(t[0], t[1]);
    part[2 * (size_t)blockIdx.x + 1] = make_double2(t[2], t[3]);
  }
}

// one CTA per timeslice: corr[p][trel] from the partials of timeslice t
__global__ void k_nucleon_timeslices(const double2* __restrict__ part, int per_t, int T, int t0, int bc3,
                                     double2* __restrict__ corr) {
  const int t = blockIdx.x;
  __shared__ double2 sh[2][256];
  double2 ap = make_double2(0, 0), am = make_double2(0, 0);
  for (int k = threadIdx.x; k < per_t; k += blockDim.x) {
    double2 p = part[2 * ((size_t)t * per_t + k)], m = part[2 * ((size_t)t * per_t + k) + 1];
    ap.x += p.x; ap.y += p.y; am.x += m.x; am.y += m.y;
  }
  sh[0][threadIdx.x] = ap;
  sh[1][threadIdx.x] = am;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      sh[0][threadIdx.x].x += sh[0][threadIdx.x + st].x; sh[0][threadIdx.x].y += sh[0][threadIdx.x + st].y;
      sh[1][threadIdx.x].x += sh[1][threadIdx.x + st].x; sh[1][threadIdx.x].y += sh[1][threadIdx.x + st].y;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    int trel = (t - t0 + T) % T;
    double sg = (t < t0) ? (double)bc3 : 1.0;
    corr[trel] = make_double2(sg * sh[0][0].x, sg * sh[0][0].y);
    corr[T + trel] = make_double2(sg * sh[1][0].x, sg * sh[1][0].y);
  }
}

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double2* g_scratch_addr[kMaxDevices] = {};

// Device address of the static scratch on the current device.  The first call
// on a device resolves it with cudaGetSymbolAddress (the host-side name of the
// array is not a device address) and sets the kernels' shared-memory limit.
qcd_status scratch_on_current_device(double2** out) {
  int dev = 0;
  QCD_CUDA_OK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    qcd_set_error("device ordinal %d out of range", dev);
    return QCD_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    QCD_CUDA_OK(cudaGetSymbolAddress(&p, g_nucleon_scratch));
    QCD_CUDA_OK(cudaFuncSetAttribute(k_nucleon_canonical<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(144 * 32 * sizeof(Cplx<double>))));
    QCD_CUDA_OK(cudaFuncSetAttribute(k_nucleon_canonical<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(144 * 32 * sizeof(Cplx<float>))));
    g_scratch_addr[dev] = (double2*)p;
  }
  *out = g_scratch_addr[dev];
  return QCD_OK;
}

}  // namespace

extern "C" qcd_status qcd_nucleon_2pt_noalloc(const int dims[4], int time_bc, const double* prop, const int src[4],
                                              double* corr, int precision, void* cuda_stream) {
  if (!dims || !prop || !src || !corr) {
    qcd_set_error("null argument");
    return QCD_ERR_ARG;
  }
  long long V = 1;
  for (int mu = 0; mu < 4; mu++) {
    if (dims[mu] < 2) {
      qcd_set_error("lattice extent %d must be >= 2", dims[mu]);
      return QCD_ERR_ARG;
    }
    if (src[mu] < 0 || src[mu] >= dims[mu]) {
      qcd_set_error("source outside the lattice");
      return QCD_ERR_ARG;
    }
    V *= dims[mu];
  }
  if (time_bc != 1 && time_bc != -1) {
    qcd_set_error("time_bc must be +1 or -1");
    return QCD_ERR_ARG;
  }
  if (precision != QCD_PREC_F64 && precision != QCD_PREC_F32) {
    qcd_set_error("unknown precision");
    return QCD_ERR_ARG;
  }
  const int L3 = dims[1] * dims[2] * dims[3];
  int ns = 32;
  while (L3 % ns) ns >>= 1;
  const long long nb = V / ns;
  if (nb > QCD_NOALLOC_MAX_CTAS) {
    qcd_set_error("lattice too large for the fixed scratch of qcd_nucleon_2pt_noalloc: %lld sites in %lld groups of "
                  "%d > %d groups (at most %d sites with a spatial volume divisible by 32)",
                  V, nb, ns, QCD_NOALLOC_MAX_CTAS, 32 * QCD_NOALLOC_MAX_CTAS);
    return QCD_ERR_ARG;
  }
  double2* scratch = nullptr;
  QCD_TRY(scratch_on_current_device(&scratch));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int T = dims[0];
  // every partial slot read below is written first by its CTA: nothing to clear
  if (precision == QCD_PREC_F64)
    k_nucleon_canonical<double><<<(unsigned)nb, 6 * ns, 144 * ns * sizeof(Cplx<double>), st>>>(
        (const double2*)prop, (int)V, ns, scratch);
  else
    k_nucleon_canonical<float><<<(unsigned)nb, 6 * ns, 144 * ns * sizeof(Cplx<float>), st>>>(
        (const double2*)prop, (int)V, ns, scratch);
  QCD_CUDA_OK(cudaGetLastError());
  k_nucleon_timeslices<<<T, 256, 0, st>>>(scratch, (int)(nb / T), T, src[0], time_bc * time_bc * time_bc,
                                          (double2*)corr);
  QCD_CUDA_OK(cudaGetLastError());
  return QCD_OK;
}
