// Little Dirac operator (Sec. 2.2, eq. little) on the fifth-generation
// tensor cores: for every deflation block b the nine N_s x N_s couplings
//   A[b][p][k][j] = sum_{y in b, spin-colour} conj(phi_k(y)) X_{p,j}(y),
// X_0 = the block-internal part of D phi_j, X_{1+2mu} / X_{2+2mu} = the hops
// across the block's +mu / -mu face (d->Y parts, face sites selected), are one
// real GEMM per block:
//   Phi = P + iQ, X = R + iS:  Re A = P^T R + Q^T S,  Im A = P^T S - Q^T R,
//   D[m][n] = sum_K Xrow_m(K) Brow_n(K),  m = (p, j, {R, S}), n = ({P, Q}, k),
// K running over the block's (site, spin-colour) entries.  tcgen05.mma
// (kind::tf32, M = 128, N = 2 ns_pad, K = 8 per instruction) with FP32
// accumulators in tensor memory; operands staged in shared memory in the
// canonical K-major layout without swizzle (core matrices of 8 rows x 16 bytes).
// Each FP32 operand x is split as x = hi + lo with hi = x truncated to the 19
// bits the tensor core reads and lo = x - hi (exact), and the product is
// hi*hi + hi*lo + lo*hi (error of order 2^-21 relative, the FP32 level of the
// FP32 fields).  Each chunk's accumulator is read with tcgen05.ld and added to
// a compensated FP32 sum (TwoSum, sum and error kept apart), widened to FP64
// at the end; A is stored in FP64.
//
// One CTA of 128 threads per (block, 128-row tile); one elected thread issues
// the MMAs and commits them to an mbarrier; all waits on it are bounded (on
// timeout the kernel records an error, frees its tensor memory and returns).
// The staged operands are double-buffered so that staging overlaps the MMAs.
#include <stdint.h>

#include "qcd_internal.cuh"

namespace {

constexpr int TC_THREADS = 128;
constexpr int KC = 24;                 // K entries per staged chunk (2 sites x 12)
constexpr int KG = KC / 4;             // core matrices along K per chunk
constexpr int WAIT_LIMIT = 1 << 20;     // polls of ~64 ns: about 70 ms before a wait gives up

__device__ inline uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// descriptor of a K-major, non-swizzled operand tile in shared memory
__device__ inline uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;              // descriptor version
  return d;                            // base offset 0, no swizzle
}

// instruction descriptor: kind::tf32, FP32 accumulate, both operands K-major
__host__ __device__ inline uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ inline float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// byte offset of element (row, k) of a staged operand: core matrix
// (row / 8, k / 4) at ((row / 8) * KG + k / 4) * 128, row (row % 8) * 16, element (k % 4) * 4
__device__ inline uint32_t stage_off(int row, int k) {
  return (uint32_t)(((row >> 3) * KG + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

__device__ inline bool mbar_wait(uint32_t bar, uint32_t phase) {
  for (int i = 0; i < WAIT_LIMIT; i++) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase)
        : "memory");
    if (done) return true;
    __nanosleep(64);
  }
  return false;
}

struct TcGeom {
  int b[4], nb[4], vb;
};

__device__ inline int tc_site(const TcGeom& bg, const Geom& g, int blk, int l, int lc[4]) {
  int bc[4];
  bc[1] = blk % bg.nb[1];
  int r = blk / bg.nb[1];
  bc[2] = r % bg.nb[2];
  r /= bg.nb[2];
  bc[3] = r % bg.nb[3];
  bc[0] = r / bg.nb[3];
  r = l;
  lc[1] = r % bg.b[1]; r /= bg.b[1];
  lc[2] = r % bg.b[2]; r /= bg.b[2];
  lc[3] = r % bg.b[3];
  lc[0] = r / bg.b[3];
  int c[4];
  for (int mu = 0; mu < 4; mu++) c[mu] = bc[mu] * bg.b[mu] + lc[mu];
  return ((c[0] * g.L[3] + c[3]) * g.L[2] + c[2]) * g.L[1] + c[1];
}

// Stage the 12 spin-colour components of one site of one field as TF32 head
// and remainder: x[q] holds components 2q, 2q + 1 (re, im, re, im); the real
// parts go to row r_re, the imaginary parts to row r_im, at K entries
// e0 .. e0 + 11.
__device__ inline void stage_site(unsigned char* hi, unsigned char* lo, int r_re, int r_im, int e0,
                                  const float4 (&x)[6]) {
#pragma unroll
  for (int c = 0; c < 2; c++) {
    const int row = c ? r_im : r_re;
#pragma unroll
    for (int g = 0; g < 3; g++) {   // K entries e0 + 4 g .. e0 + 4 g + 3: components 4 g .. 4 g + 3
      const float4 a = x[2 * g], b = x[2 * g + 1];
      const float4 v = c ? make_float4(a.y, a.w, b.y, b.w) : make_float4(a.x, a.z, b.x, b.z);
      const float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
      const uint32_t off = stage_off(row, e0 + 4 * g);
      *(float4*)(hi + off) = h;
      *(float4*)(lo + off) = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
    }
  }
}

// CTA (block b, tile t): rows 128 t .. 128 t + 127 of the X side against all
// N = 2 NSP columns of the Phi side.  The accumulator in tensor memory holds
// one chunk (KC entries of K, 9 MMAs); after each chunk every thread adds its
// row's N values to its compensated sums and the next chunk starts a fresh
// accumulation, so no FP32 accumulator sums more than one chunk (the tensor
// core's accumulation rounds toward zero by up to an FP32 ulp per MMA, which
// over the whole K of a 4^4 block biased the sums by 5e-5 relative).
// The operands are double-buffered: chunk ch + 1 is staged while the MMAs of
// chunk ch run.  Staging works in tasks of one row pair (the real and the
// imaginary row of one field) and one of the chunk's two sites: six 16-byte
// loads of the site's components feed both rows.
template <int NSP>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_dfl_little_tc(const char* __restrict__ phi, const char* __restrict__ Y, double* __restrict__ A, Geom g,
                    TcGeom bg, int ns, int tmem_cols, int* __restrict__ err) {
  constexpr int N = 2 * NSP;           // real columns of the Phi side
  constexpr int M = 9 * 2 * NSP;       // real rows of the X side
  constexpr size_t A_BYTES = 128 * KC * 4, B_BYTES = N * KC * 4;
  constexpr size_t BUF = 2 * (A_BYTES + B_BYTES);   // hi and lo of both operands
  constexpr int XTASKS = 64 * 2, TASKS = XTASKS + NSP * 2;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int blk = blockIdx.x, tile = blockIdx.y;
  const size_t fb = FieldsF::spinor_bytes * (size_t)g.V;
  // a CTA started after another one gave up does no work (uniform per CTA)
  if (*(volatile int*)err) return;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = tmem_base;
  const uint32_t idesc = instr_desc(128, N);
  const uint32_t bar = smem_u32(&mbar);
  bool ok = true;
  uint32_t phase = 0;
  // compensated FP32 sums of the chunks' results (sum + running error, TwoSum
  // per chunk): FP64 additions run at 1/64 of the FP32 rate on this GPU
  float sum[N], cmp[N];
#pragma unroll
  for (int q = 0; q < N; q++) sum[q] = cmp[q] = 0.f;

  // stage chunk ch (sites 2 ch, 2 ch + 1 of the block) into buffer buf
  auto stage = [&](int ch, int buf) {
    unsigned char* a_hi = smem_raw + buf * BUF;
    unsigned char* a_lo = a_hi + A_BYTES;
    unsigned char* b_hi = a_lo + A_BYTES;
    unsigned char* b_lo = b_hi + B_BYTES;
    for (int t = tid; t < TASKS; t += TC_THREADS) {
      const int site = t & 1;
      int lc[4];
      const int s = tc_site(bg, g, blk, 2 * ch + site, lc);
      float4 x[6];
      bool on = false;
      const char* src = nullptr;
      int r0;
      unsigned char *hi, *lo;
      if (t < XTASKS) {
        r0 = 2 * (t >> 1);                    // rows r0 (real part), r0 + 1 (imaginary part) of the tile
        hi = a_hi;
        lo = a_lo;
        const int grow = tile * 128 + r0;
        const int j = (grow >> 1) % NSP, p = (grow >> 1) / NSP;
        if (grow < M && j < ns) {
          int part = 0;
          on = true;
          if (p > 0) {
            const int mu = (p - 1) >> 1;
            // lc[mu], b[mu] by selects (no local-memory indexing)
            const int lm = mu == 0 ? lc[0] : mu == 1 ? lc[1] : mu == 2 ? lc[2] : lc[3];
            const int bm = mu == 0 ? bg.b[0] : mu == 1 ? bg.b[1] : mu == 2 ? bg.b[2] : bg.b[3];
            on = ((p - 1) & 1) == 0 ? lm == bm - 1 : lm == 0;
            part = 1 + mu;
          }
          src = Y + ((size_t)part * ns + j) * fb;
        }
      } else {
        const int k = (t - XTASKS) >> 1;      // Phi rows k (real part) and NSP + k (imaginary part)
        r0 = k;
        hi = b_hi;
        lo = b_lo;
        on = k < ns;
        src = phi + (size_t)k * fb;
      }
#pragma unroll
      for (int q = 0; q < 6; q++)
        x[q] = on ? __ldg((const float4*)src + (size_t)q * g.V + s) : make_float4(0.f, 0.f, 0.f, 0.f);
      // X side: real and imaginary rows neighbours; Phi side: NSP apart
      if (t < XTASKS)
        stage_site(hi, lo, r0, r0 + 1, 12 * site, x);
      else
        stage_site(hi, lo, r0, r0 + NSP, 12 * site, x);
    }
  };

  const int nchunks = bg.vb * 12 / KC;
  stage(0, 0);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  for (int ch = 0; ch < nchunks && ok; ch++) {
    const int buf = ch & 1;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned char* a_hi = smem_raw + buf * BUF;
      const unsigned char* a_lo = a_hi + A_BYTES;
      const unsigned char* b_hi = a_lo + A_BYTES;
      const unsigned char* b_lo = b_hi + B_BYTES;
      for (int ks = 0; ks < KC / 8; ks++)
        for (int term = 0; term < 3; term++) {
          const unsigned char* aop = term == 2 ? a_lo : a_hi;
          const unsigned char* bop = term == 1 ? b_lo : b_hi;
          const uint64_t ad = smem_desc(smem_u32(aop) + (uint32_t)(2 * ks * 128), 128, KG * 128);
          const uint64_t bd = smem_desc(smem_u32(bop) + (uint32_t)(2 * ks * 128), 128, KG * 128);
          const uint32_t accum = (ks > 0 || term > 0) ? 1u : 0u;   // each chunk starts a fresh sum
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tbase),
              "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
              : "memory");
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                   : "memory");
    }
    // the next chunk goes into the other buffer, whose MMAs completed in the
    // previous iteration, while this chunk's MMAs run
    if (ch + 1 < nchunks) stage(ch + 1, buf ^ 1);
    // this chunk's MMAs complete before the accumulator is read and before
    // their buffer is staged again
    const bool done = mbar_wait(bar, phase);
    phase ^= 1u;
    if (done) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int cb = 0; cb < N; cb += 16) {
        uint32_t r[16];
        const uint32_t ta = tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)cb;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(ta)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int q = 0; q < 16; q++) {
          const float x = __uint_as_float(r[q]), a = sum[cb + q];
          const float t = a + x, bp = t - a;
          cmp[cb + q] += (a - (t - bp)) + (x - bp);   // the rounding error of a + x, exactly
          sum[cb + q] = t;
        }
      }
    }
    // the staged writes of the next chunk are visible to the tensor core and
    // the accumulator reads are done before the next MMAs; every thread leaves
    // the loop together if any wait gave up
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    ok = __syncthreads_and(done) != 0;
  }
  if (!ok) {
    if (tid == 0) atomicExch(err, 1);
    mbar_wait(bar, phase ^ 1u);   // a last bounded wait for MMAs still in flight
  }

  if (ok) {
    // rows (p, j, R) and (p, j, S) are neighbouring lanes: Re A = D[R][k] + D[S][NSP + k],
    // Im A = D[S][k] - D[R][NSP + k]; sum and error widened to FP64 once
    const int row = tile * 128 + 32 * warp + lane;
    const int c = row & 1, j = (row >> 1) % NSP, p = (row >> 1) / NSP;
#pragma unroll
    for (int k = 0; k < NSP; k++) {
      const double mine = (double)sum[k] + (double)cmp[k];
      const double other = __shfl_xor_sync(0xffffffffu, (double)sum[NSP + k] + (double)cmp[NSP + k], 1);
      const double v = c == 0 ? mine + other : mine - other;
      if (p < 9 && j < ns && k < ns) A[((((size_t)blk * 9 + p) * ns + k) * ns + j) * 2 + c] = v;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(tmem_cols) : "memory");
}

}  // namespace

// A (FP64 [nblk][9][ns][ns] complex) from the deflation fields phi and the
// parts Y of D phi (FP32 internal layouts), on the tensor cores.  err: device
// int, set to 1 if a wait on the tensor cores timed out.
qcd_status dfl_little_tc(qcd_ctx* c, const void* phi, const void* Y, double* A, const int b[4], int ns, int* err) {
  TcGeom bg;
  bg.vb = 1;
  int nblk = 1;
  for (int mu = 0; mu < 4; mu++) {
    bg.b[mu] = b[mu];
    bg.nb[mu] = c->g.L[mu] / b[mu];
    bg.vb *= b[mu];
    nblk *= bg.nb[mu];
  }
  if ((bg.vb * 12) % KC != 0 || ns < 1 || ns > 32) {
    qcd_set_error("tensor-core little Dirac build needs 12 x block volume divisible by %d and 1 <= ns <= 32", KC);
    return QCD_ERR_ARG;
  }
  const int nsp = (ns + 7) / 8 * 8;
  const int M = 9 * 2 * nsp, N = 2 * nsp;
  const int ntiles = (M + 127) / 128;
  const int cols = N < 32 ? 32 : N;                              // N is 16, 32, 48 or 64
  const int tmem_cols = cols == 48 ? 64 : cols;                  // a power of two >= 32
  const size_t smem = (size_t)(128 + N) * KC * 4 * 2 * 2;   // hi + lo, double-buffered
  const dim3 grid((unsigned)nblk, (unsigned)ntiles);
  ProfScope ps(c, FAM_DFL, (double)spinor_bytes(c, QCD_PREC_F32) * ns * 6,
               2.0 * nblk * (double)M * N * bg.vb * 12 * 3);
  switch (nsp) {
#define TC_CASE(X)                                                                                              \
  case X:                                                                                                       \
    QCD_CUDA_OK(cudaFuncSetAttribute(k_dfl_little_tc<X>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
    k_dfl_little_tc<X><<<grid, TC_THREADS, smem, c->stream>>>((const char*)phi, (const char*)Y, A, c->g, bg, ns,   \
                                                              tmem_cols, err);                                   \
    break;
    TC_CASE(8)
    TC_CASE(16)
    TC_CASE(24)
    TC_CASE(32)
#undef TC_CASE
  }
  QCD_CUDA_OK(cudaGetLastError());
  return QCD_OK;
}
