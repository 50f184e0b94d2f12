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
// writes the correlator to device memory.  The kernels are the ones of
// qcd_nucleon_2pt (nucleon_kernels.cuh), instantiated for the canonical
// layout.
#include <mutex>

#include "nucleon_kernels.cuh"

// Largest number of partial sums held in the static scratch: two (P+ and P-)
// per CTA of 32 sites, i.e. V <= 32 * 131072 = 4,194,304 sites (e.g. 32^3 x 128
// or 40^3 x 64).  4 MiB of device memory.
#define QCD_NOALLOC_MAX_CTAS 131072

static __device__ __align__(256) double2 g_nucleon_scratch[2 * QCD_NOALLOC_MAX_CTAS];

namespace {

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
    QCD_CUDA_OK(cudaFuncSetAttribute(nucleon::k_sites<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(144 * 32 * sizeof(Cplx<double>))));
    QCD_CUDA_OK(cudaFuncSetAttribute(nucleon::k_sites<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
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
    V *= dims[mu];   // < 2^31 before, so < 2^62 here
    if (V >= (1LL << 31)) {
      qcd_set_error("lattice volume too large (T*X*Y*Z must be < 2^31)");
      return QCD_ERR_ARG;
    }
  }
  if (time_bc != 1 && time_bc != -1) {
    qcd_set_error("time_bc must be +1 or -1");
    return QCD_ERR_ARG;
  }
  if (precision != QCD_PREC_F64 && precision != QCD_PREC_F32) {
    qcd_set_error("unknown precision");
    return QCD_ERR_ARG;
  }
  const long long L3 = (long long)dims[1] * dims[2] * dims[3];
  const int ns = nucleon::sites_per_cta(L3);
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
  const int threads = nucleon::cta_threads(ns);
  if (precision == QCD_PREC_F64)
    nucleon::k_sites<double, true><<<(unsigned)nb, threads, 144 * ns * sizeof(Cplx<double>), st>>>(
        (const double2*)prop, (int)V, ns, scratch);
  else
    nucleon::k_sites<float, true><<<(unsigned)nb, threads, 144 * ns * sizeof(Cplx<float>), st>>>(
        (const double2*)prop, (int)V, ns, scratch);
  QCD_CUDA_OK(cudaGetLastError());
  nucleon::k_timeslices<<<T, 256, 0, st>>>(scratch, (int)(nb / T), T, src[0], time_bc * time_bc * time_bc,
                                           (double2*)corr);
  QCD_CUDA_OK(cudaGetLastError());
  return QCD_OK;
}
