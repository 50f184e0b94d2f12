// Kernels of the nucleon two-point function (eq. Nop and the P+- projections
// of Sec. 2.3), shared by qcd_nucleon_2pt (internal propagator layout) and
// qcd_nucleon_2pt_noalloc (canonical layout).
//
// N_alpha = eps^{abc} (u^a^T G d^b) u^c_alpha, G = C g5, C = g0 g2; with u = d
// and one point-source propagator S (12x12 per site, S^{a a'}_{alpha alpha'}),
// the Wick contractions give
//   G(x) = eps^{abc} eps^{a'b'c'} { S^{cc'} tr[S^{aa'T} G S^{bb'} G']
//                                   - S^{ca'} G'^T S^{bb'T} G^T S^{ac'} },
// G' = g0 G^+ g0^T.  In the chiral basis G = diag(J, J), J = [[0,-1],[1,0]],
// and G' = -G, so both are signed permutations: G_{b, b^1} = g(b) and
// G'_{b^1, b} = g(b) with g(b) = -1 for even b, +1 for odd b.  Hence
//   tr[S^{aa'T} G S^{bb'} G'] = sum_{b,b'} g(b) g(b') S^{aa'}_{b b'} S^{bb'}_{b^1 b'^1}
//   (G'^T S^{bb'T} G^T)_{ij} = g(i) g(j) S^{bb'}_{j^1 i^1}
// and with P+- = (1 +- g0)/2, tr[P+- Z] = (1/2) sum_l (Z_{ll} -+ Z_{l^2, l}).
//
// Layout: 6 threads per site, one per sink colour permutation (a,b,c), each
// summing over the 6 source permutations.  A CTA covers NS consecutive sites
// of one timeslice (NS a power of two dividing the spatial volume, so a CTA
// never straddles two timeslices); the propagator of those sites is staged
// in shared memory (the 144 complex entries of a site are read by its 6
// threads).  The CTA has 6 NS threads rounded up to whole warps; the padding
// threads stage but contribute zero to the sums, so every warp of the
// shuffle reduction is full.  The CTA's sum over its sites is written to a
// partial; a second kernel sums the partials of each timeslice in a fixed
// order, re-references the time to the source and applies the boundary sign
// of wrapped sink times.
#pragma once

#include "qcd_internal.cuh"

// an unnamed namespace: each translation unit that includes this header
// gets its own copy of the kernels and of the constant table
namespace nucleon {
namespace {

__constant__ int c_perm[6][4] = {  // a, b, c, sign
    {0, 1, 2, 1}, {1, 2, 0, 1}, {2, 0, 1, 1}, {0, 2, 1, -1}, {2, 1, 0, -1}, {1, 0, 2, -1}};

template <typename R>
__device__ inline Cplx<R> Sget(const Cplx<R>* S_s, int ns, int i, int al, int a, int alp, int ap) {
  return S_s[((3 * al + a) * 12 + 3 * alp + ap) * ns + i];
}

template <typename R>
__device__ inline R gsign(int b) { return (b & 1) ? (R)1 : (R)-1; }

// threads of a CTA covering ns sites: 6 ns rounded up to a multiple of 32
inline int cta_threads(int ns) { return (6 * ns + 31) & ~31; }

// CANONICAL = true: prop is [rhs][site][spin][colour] complex FP64 (the C-ABI
// layout); false: the internal FP64 spinor layout double2 [rhs][12][V].
template <typename R, bool CANONICAL>
__global__ void k_sites(const double2* __restrict__ prop, int V, int ns, double2* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cplx<R>* S_s = (Cplx<R>*)smem_raw;
  const int s0 = blockIdx.x * ns;
  // stage: entry e = comp*12 + rhs of site s0 + i
  for (int idx = threadIdx.x; idx < 144 * ns; idx += blockDim.x) {
    const int i = idx % ns, e = idx / ns;
    const int comp = e / 12, rhs = e - comp * 12;
    const double2 v = CANONICAL ? prop[((size_t)rhs * V + s0 + i) * 12 + comp]
                                : prop[((size_t)rhs * 12 + comp) * V + s0 + i];
    S_s[e * ns + i] = cmk((R)v.x, (R)v.y);
  }
  __syncthreads();

  Cplx<R> accp = cmk((R)0, (R)0), accm = cmk((R)0, (R)0);
  if (threadIdx.x < 6 * ns) {
    const int i = threadIdx.x % ns;
    const int pq = threadIdx.x / ns;   // sink permutation 0..5
    const int a = c_perm[pq][0], b = c_perm[pq][1], c = c_perm[pq][2];
    const R eps = (R)c_perm[pq][3];
#pragma unroll 1
    for (int q = 0; q < 6; q++) {
      const int ap = c_perm[q][0], bp = c_perm[q][1], cp = c_perm[q][2];
      const R ee = eps * (R)c_perm[q][3];
      // T = tr[S^{aa'T} G S^{bb'} G']
      Cplx<R> T = cmk((R)0, (R)0);
#pragma unroll
      for (int be = 0; be < 4; be++)
#pragma unroll
        for (int bq = 0; bq < 4; bq++) {
          const Cplx<R> x = Sget(S_s, ns, i, be, a, bq, ap) * Sget(S_s, ns, i, be ^ 1, b, bq ^ 1, bp);
          T = T + (gsign<R>(be) * gsign<R>(bq)) * x;
        }
      // tr[P+- S^{cc'}]
      Cplx<R> d = cmk((R)0, (R)0), o = cmk((R)0, (R)0);
#pragma unroll
      for (int l = 0; l < 4; l++) {
        d = d + Sget(S_s, ns, i, l, c, l, cp);
        o = o + Sget(S_s, ns, i, l ^ 2, c, l, cp);
      }
      const Cplx<R> t1p = T * ((R)0.5 * (d - o)), t1m = T * ((R)0.5 * (d + o));
      // Y = S^{ca'} M, M_{kj} = g(k) g(j) S^{bb'}_{j^1 k^1}
      Cplx<R> Y[4][4];
#pragma unroll
      for (int ii = 0; ii < 4; ii++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
          Cplx<R> y = cmk((R)0, (R)0);
#pragma unroll
          for (int k = 0; k < 4; k++)
            y = y + (gsign<R>(k) * gsign<R>(j)) *
                        (Sget(S_s, ns, i, ii, c, k, ap) * Sget(S_s, ns, i, j ^ 1, b, k ^ 1, bp));
          Y[ii][j] = y;
        }
      // tr[P+- Y S^{ac'}] = (1/2) sum_{l,k} (Y_{lk} -+ Y_{l^2 k}) S^{ac'}_{kl}
      Cplx<R> zd = cmk((R)0, (R)0), zo = cmk((R)0, (R)0);
#pragma unroll
      for (int l = 0; l < 4; l++)
#pragma unroll
        for (int k = 0; k < 4; k++) {
          const Cplx<R> sv = Sget(S_s, ns, i, k, a, l, cp);
          zd = zd + Y[l][k] * sv;
          zo = zo + Y[l ^ 2][k] * sv;
        }
      const Cplx<R> t2p = (R)0.5 * (zd - zo), t2m = (R)0.5 * (zd + zo);
      accp = accp + ee * (t1p - t2p);
      accm = accm + ee * (t1m - t2m);
    }
  }
  // CTA sum (fixed order): warp shuffles over full warps, then one thread
  // over the warp sums
  __shared__ double red[4][32];
  double v[4] = {(double)accp.re, (double)accp.im, (double)accm.re, (double)accm.im};
#pragma unroll
  for (int k = 0; k < 4; k++)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
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

// one CTA of 256 threads per timeslice: corr[p][trel] = sign * sum of the
// partials of timeslice t
__global__ void k_timeslices(const double2* __restrict__ part, int per_t, int T, int t0, int bc3,
                             double2* __restrict__ corr) {
  const int t = blockIdx.x;
  __shared__ double2 sh[2][256];
  double2 ap = make_double2(0, 0), am = make_double2(0, 0);
  for (int k = threadIdx.x; k < per_t; k += blockDim.x) {
    const double2 p = part[2 * ((size_t)t * per_t + k)], m = part[2 * ((size_t)t * per_t + k) + 1];
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
    const int trel = (t - t0 + T) % T;
    const double sg = (t < t0) ? (double)bc3 : 1.0;
    corr[trel] = make_double2(sg * sh[0][0].x, sg * sh[0][0].y);
    corr[T + trel] = make_double2(sg * sh[1][0].x, sg * sh[1][0].y);
  }
}

// sites per CTA: the largest power of two <= 32 dividing the spatial volume
inline int sites_per_cta(long long L3) {
  int ns = 32;
  while (L3 % ns) ns >>= 1;
  return ns;
}

}  // namespace
}  // namespace nucleon
