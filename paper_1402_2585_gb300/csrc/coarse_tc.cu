// Little Dirac operator on the tensor cores (tcgen05), for 1..16 right-hand
// sides at once:  Y_a = sum_{l in {-1,0,1}^4} A^{a,a+l} X_{a+l}  (Sec. 5.1).
//
// The complex Nvec x Nvec block A^{a,l} enters the MMA as a real matrix with
// interleaved rows m = 2j + ri (ri = 0: Re A_jk, ri = 1: Im A_jk), so
//   D[2j+0][c] = sum_k Re A_jk B[k][c],   D[2j+1][c] = sum_k Im A_jk B[k][c]
// and the complex product follows in the epilogue from the columns of B,
// which hold, per right-hand side r, the four real vectors
//   c = 4r + {0: Re X_hi, 1: Im X_hi, 2: Re X_lo, 3: Im X_lo}.
// X_hi + X_lo is the FP32 vector scaled by a power of two per right-hand side
// (largest entry in [2^13, 2^14)) and split into two FP16 parts, so the
// product carries about 22 significant bits of X, with A in FP16 and FP32
// accumulation.  Re Y = P_even - Q_odd, Im Y = Q_even + P_odd, where P = D[.,
// Re X_hi] + D[., Re X_lo] and Q = D[., Im X_hi] + D[., Im X_lo] of the two
// rows of coefficient j (adjacent TMEM lanes, exchanged by one shuffle).
//
// Every coarse site's 81 blocks carry one power-of-two scale (largest entry in
// [2^13, 2^14)), so the far couplings, many orders of magnitude below the
// diagonal block, stay in FP16's normal range; the epilogue removes it.  An FP32
// operator is split into FP16 hi + lo parts (about 22 significant bits) that
// enter as two MMAs against the same B tile; an FP16 operator is one part.
//
// With Nvec <= 32 a block has at most 64 rows, so two coarse sites share one
// M = 128 MMA (rows 0..63 site a0, 64..127 site a1) against B = [B_{a0+l} |
// B_{a1+l}]; the two off-diagonal quadrants of D are discarded.  Above 32 one
// site per MMA: its 2 Nvec rows are stored and the MMA's remaining rows are
// discarded.
// K = Nvec padded to a multiple of 16.  Both operands are pre-tiled in global
// memory in the no-swizzle K-major core-matrix layout, so every stage of the
// pipeline is filled by plain bulk copies: the A blocks of the sites (the HBM
// stream, exactly the operator's bytes) and the B tiles of their neighbours
// (L2-resident).
//
// Pipeline per CTA (persistent, up to two CTAs per SM): warp 0 issues the
// copies into a ring of stages, warp 1 issues the MMAs (one accumulator in
// tensor memory per site pair) and releases stages through tcgen05.commit,
// warps 2..5 read the accumulator (one TMEM lane quarter each), combine,
// unscale and store Y and the per-right-hand-side <X, Y>.
#include <algorithm>
#include <cstring>

#include "coarse.cuh"
#include "tc.cuh"

namespace hdcg {

namespace {

constexpr int TC_THREADS = 192;
constexpr int TC_RPMAX = RMAX;                 // right-hand sides per launch
constexpr uint32_t TC_RING_BYTES = 96 * 1024;  // two CTAs per SM
constexpr uint32_t TC_RING_BYTES_1 = 192 * 1024;  // one CTA per SM

int device_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    HDCG_CUDA(cudaGetDevice(&dev));
    HDCG_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  }
  return n;
}

void set_smem(const void* fn, size_t bytes) {
  HDCG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

// power-of-two scale that brings max|x| into [2^13, 2^14): exponent e, clamped
__device__ __forceinline__ int scale_exp(unsigned maxbits) {
  if (maxbits == 0) return 0;
  const int E = (int)((maxbits >> 23) & 0xffu);
  return min(126, max(-126, 140 - E));
}
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

}  // namespace

TcGeom tc_geom(int nvec, int R, int parts, uint32_t ring_bytes) {
  HDCG_REQUIRE(nvec >= 1 && nvec <= 64, HDCG_ERR_ARG, "tensor-core coarse operator needs Nvec <= 64");
  HDCG_REQUIRE(R >= 1 && R <= TC_RPMAX, HDCG_ERR_ARG, "1..16 right-hand sides");
  TcGeom g;
  // two sites share an MMA for Nvec <= 32 (exactly its 128 rows at Nvec 32);
  // one site per MMA above that, with the compact layout below, which copies
  // only the operator's bytes
  g.sites = nvec <= 32 ? 2 : 1;
  g.MS = 128 / g.sites;
  g.Kp = (nvec + 15) / 16 * 16;
  const int q = g.sites == 2 ? 2 : 4;   // keeps N = sites * 4 Rp a multiple of 16
  g.Rp = (R + q - 1) / q * q;
  g.NS = 4 * g.Rp;
  g.NMMA = g.sites * g.NS;
  g.ncols = 32;
  while (g.ncols < g.NMMA) g.ncols *= 2;
  g.b_bytes = (uint32_t)g.NS * g.Kp * 2;
  g.parts = parts;
  if (g.sites == 2) {
    // two sites share the M = 128 rows: each block stored whole (MS x Kp),
    // core matrices K-adjacent 128 B apart and M-adjacent 16 Kp B apart
    g.rows = g.MS;
    g.kgs = g.Kp / 8;
    g.a_gbytes = (uint32_t)g.MS * g.Kp * 2;
    g.a_sbytes = g.a_gbytes;
    g.lbo_a = 128;
    g.sbo_a = (uint32_t)g.Kp * 16;
  } else {
    // one site: only the 2 Nvec rows (in 8-row groups) and the Nvec columns
    // (in 8-wide K groups) are stored, K group by K group (M-adjacent core
    // matrices 128 B apart, K-adjacent RG 128 B apart), so a stage copies
    // exactly the operator's bytes.  The MMA reads 16 row groups and Kp / 8
    // K groups: rows past 2 Nvec come from the next K group (finite values;
    // their output rows are discarded), and the K groups past Nvec from the
    // slot's tail, which no copy writes and which stays zero (the kernel
    // clears the ring once).
    const int RG = (2 * nvec + 7) / 8;
    g.rows = 8 * RG;
    g.kgs = (nvec + 7) / 8;
    g.a_gbytes = (uint32_t)(g.kgs * RG * 128);
    g.a_sbytes = (uint32_t)(((g.Kp / 8 - 1) * RG + 16) * 128);
    g.lbo_a = (uint32_t)RG * 128u;
    g.sbo_a = 128;
  }
  g.stage_bytes = g.sites * (parts * g.a_sbytes + g.b_bytes);
  g.copy_bytes = g.sites * (parts * g.a_gbytes + g.b_bytes);
  g.stages = (int)std::min<uint32_t>(16, ring_bytes / g.stage_bytes);
  g.stages = std::max(g.stages, 2);
  return g;
}

__device__ __forceinline__ float2 a_value(const __half2* A, size_t i) { return __half22float2(A[i]); }
__device__ __forceinline__ float2 a_value(const float2* A, size_t i) { return A[i]; }

// per coarse site: scale exponent bringing the largest |Re|, |Im| of its 81 blocks into [2^13, 2^14)
template <typename AT>
__global__ void k_site_scale(const AT* __restrict__ A, int n, int* sexp) {
  const size_t a = blockIdx.x;
  const size_t per = (size_t)81 * n * n;
  float m = 0.f;
  for (size_t i = threadIdx.x; i < per; i += blockDim.x) {
    const float2 v = a_value(A, a * per + i);
    m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
  }
  __shared__ float sm[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(FULL_MASK, m, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, sm[w]);
    sexp[a] = scale_exp(__float_as_uint(fmaxf(m, sm[0])));
  }
}

// A ([a][l][k][j] complex, FP16 or FP32) -> tiled operand, one 16-byte row segment per
// thread: element (m, k) (m < rows, k < 8 kgs) of part p of block (a, l) at byte
// (blk parts + p) a_gbytes + (m/8) sbo + (k/8) lbo + (m%8) 16 + (k%8) 2; part 0 = hi,
// part 1 = lo.
template <typename AT>
__global__ void k_a_to_tc(const AT* __restrict__ A, uint4* __restrict__ Atc, size_t nblk, int n, int rows, int kgs,
                          uint32_t a_gbytes, uint32_t lbo, uint32_t sbo, int parts, const int* __restrict__ sexp) {
  const int KG = kgs;
  const size_t per = (size_t)rows * KG;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nblk * per) return;
  const size_t blk = t / per;
  const int rem = (int)(t % per);
  const int m = rem / KG, kg = rem % KG;
  const int j = m >> 1, ri = m & 1;
  const float s = pow2f(sexp[blk / 81]);
  __align__(16) __half hi[8];
  __align__(16) __half lo[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int k = kg * 8 + q;
    float x = 0.f;
    if (j < n && k < n) {
      const float2 e = a_value(A, (blk * n + k) * n + j);
      x = (ri ? e.y : e.x) * s;
    }
    hi[q] = __float2half_rn(x);
    lo[q] = __float2half_rn(x - __half2float(hi[q]));
  }
  char* dst = reinterpret_cast<char*>(Atc) + blk * parts * (size_t)a_gbytes + (size_t)(m / 8) * sbo +
              (size_t)kg * lbo + (m % 8) * 16;
  *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(hi);
  if (parts == 2) *reinterpret_cast<uint4*>(dst + a_gbytes) = *reinterpret_cast<const uint4*>(lo);
}

// X (FP32 complex [a][k][r]) -> tiled B operand of every coarse site: thread
// (a, kg, r) writes the four 16-byte rows c = 4r + part for k = 8 kg .. 8 kg + 7.
// Rows r >= R and k >= n are written as zeros, so the whole tile is defined.
__global__ void k_x_to_tc(const float2* __restrict__ x, uint4* __restrict__ xtc, size_t Vc, int n, int R, int Rp,
                          int Kp, const unsigned* __restrict__ xmax, const int* skip) {
  if (skip && *skip) return;
  const int KG = Kp / 8;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= Vc * KG * Rp) return;
  const int r = (int)(t % Rp);
  const int kg = (int)((t / Rp) % KG);
  const size_t a = t / ((size_t)Rp * KG);
  const float s = r < R ? pow2f(scale_exp(xmax[r])) : 0.f;
  __align__(16) __half v[4][8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int k = kg * 8 + q;
    float2 xv = make_float2(0.f, 0.f);
    if (r < R && k < n) xv = x[(a * n + k) * R + r];
    const float re = xv.x * s, im = xv.y * s;
    const __half rh = __float2half_rn(re), ih = __float2half_rn(im);
    v[0][q] = rh;
    v[1][q] = ih;
    v[2][q] = __float2half_rn(re - __half2float(rh));
    v[3][q] = __float2half_rn(im - __half2float(ih));
  }
  const int NS = 4 * Rp;
  char* tile = reinterpret_cast<char*>(xtc) + a * (size_t)NS * Kp * 2;
#pragma unroll
  for (int part = 0; part < 4; ++part) {
    const int c = 4 * r + part;
    *reinterpret_cast<uint4*>(tile + (size_t)(c / 8) * (Kp * 16) + kg * 128 + (c % 8) * 16) =
        *reinterpret_cast<const uint4*>(v[part]);
  }
}

// per-right-hand-side max(|Re x|, |Im x|) as float bits (atomicMax on non-negative floats)
__global__ void k_cmax(const float2* __restrict__ x, size_t ne, int R, unsigned* xmax) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  float m[RMAX];
#pragma unroll
  for (int r = 0; r < RMAX; ++r) m[r] = 0.f;
  if (t < ne)
#pragma unroll
    for (int r = 0; r < RMAX; ++r)
      if (r < R) {
        const float2 v = x[t * R + r];
        m[r] = fmaxf(fabsf(v.x), fabsf(v.y));
      }
#pragma unroll
  for (int r = 0; r < RMAX; ++r) {
    if (r >= R) break;
    float v = m[r];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(FULL_MASK, v, o));
    if ((threadIdx.x & 31) == 0 && v > 0.f) atomicMax(xmax + r, __float_as_uint(v));
  }
}

struct TcArgs {
  const uint4* Atc;
  const int* cnbr;
  const uint4* xtc;
  const unsigned* xmax;
  const float2* x;     // FP32 X for <X, Y> (nullable)
  float2* y;
  const int* skip;     // nonzero: the launch has nothing to do (nullable)
  unsigned* err;       // bit flags of expired waits
  int Vc, n, R, sites, MS, Kp, NS, stages, ncols;
  uint32_t a_gbytes, a_sbytes, lbo_a, sbo_a, b_bytes, copy_bytes, idesc;
  float shift;         // Y = (A + shift) X (needs x)
  int parts;           // 1: FP16 operator, 2: FP32 operator as FP16 hi + lo
  const int* sexp;     // per-site scale exponents of the tiled operator
};

__global__ void __launch_bounds__(TC_THREADS, 2) k_capply_tc(TcArgs g, Reduction red) {
  extern __shared__ __align__(128) unsigned char smem[];
  if (g.skip && *g.skip) return;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t stage_bytes = g.sites * (g.parts * g.a_sbytes + g.b_bytes);
  const uint32_t ring = tc::smem_u32(smem);
  // clear the ring once: the tails of the A slots that no copy writes are read
  // by the MMAs as K padding and must be zero
  for (uint32_t i = threadIdx.x; i < (uint32_t)g.stages * stage_bytes / 16u; i += blockDim.x)
    reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
  tc::fence_proxy_async_smem();
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)g.stages * stage_bytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2 * g.stages + 3);
  const uint32_t bar0 = tc::smem_u32(bars);
  const uint32_t ACC_FULL = bar0 + 8u * (2 * g.stages), ACC_EMPTY = ACC_FULL + 8u, DRAIN = ACC_FULL + 16u;
#define TC_FULL(s) (bar0 + 8u * (uint32_t)(s))
#define TC_EMPTY(s) (bar0 + 8u * (uint32_t)(g.stages + (s)))
  if (threadIdx.x == 0) {
    for (int s = 0; s < g.stages; ++s) {
      tc::mbar_init(TC_FULL(s), 1);
      tc::mbar_init(TC_EMPTY(s), 1);
    }
    tc::mbar_init(ACC_FULL, 1);
    tc::mbar_init(ACC_EMPTY, 4);
    tc::mbar_init(DRAIN, 1);
    tc::fence_mbar_init();
  }
  if (w == 1) {
    tc::tmem_alloc(tc::smem_u32(tslot), (uint32_t)g.ncols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  const int npairs = (g.Vc + g.sites - 1) / g.sites;
  double dot[RMAX];
#pragma unroll
  for (int r = 0; r < RMAX; ++r) dot[r] = 0.0;

  if (w == 0) {
    // ---- producer: bulk copies of A blocks and neighbour B tiles --------------------
    // The whole warp first fetches the pair's 81 (or 162) neighbour indices into
    // shared memory in one round trip; lane 0 then issues the copies without a
    // dependent global load in front of every stage.
    __shared__ int snb[2 * 81];
    uint32_t it = 0;
    bool ok = true;
    for (int p = blockIdx.x; ok && p < npairs; p += gridDim.x) {
      const int s0 = p * g.sites;
      const int s1 = min(s0 + 1, g.Vc - 1);
      for (int q = lane; q < g.sites * 81; q += 32)
        snb[q] = __ldg(g.cnbr + (size_t)(q < 81 ? s0 : s1) * 81 + q % 81);
      __syncwarp();
      if (lane == 0) {
        for (int l = 0; l < 81; ++l, ++it) {
          const int s = (int)(it % (uint32_t)g.stages);
          const uint32_t ph = (it / (uint32_t)g.stages) & 1u;
          if (!tc::mbar_wait(TC_EMPTY(s), ph ^ 1u)) {
            ok = false;
            atomicOr(g.err, 1u);
            break;
          }
          tc::mbar_arrive_expect_tx(TC_FULL(s), g.copy_bytes);
          const uint32_t dst = ring + (uint32_t)s * stage_bytes;
          // stage: [part 0: site 0, site 1][part 1: site 0, site 1][B site 0][B site 1]
          for (int pp = 0; pp < g.parts; ++pp)
            for (int si = 0; si < g.sites; ++si) {
              const size_t blk = (size_t)(si ? s1 : s0) * 81 + l;
              tc::bulk_g2s(dst + (pp * g.sites + si) * g.a_sbytes,
                           reinterpret_cast<const char*>(g.Atc) + (blk * g.parts + pp) * g.a_gbytes, g.a_gbytes,
                           TC_FULL(s));
            }
          for (int si = 0; si < g.sites; ++si) {
            const int nb = snb[si * 81 + l];
            tc::bulk_g2s(dst + g.sites * g.parts * g.a_sbytes + si * g.b_bytes,
                         reinterpret_cast<const char*>(g.xtc) + (size_t)nb * g.b_bytes, g.b_bytes, TC_FULL(s));
          }
        }
      }
      ok = __shfl_sync(FULL_MASK, ok ? 1 : 0, 0) != 0;
      __syncwarp();   // lane 0 is done with snb before the next pair overwrites it
    }
    if (lane == 0) {
      // every copy issued has to land before the CTA exits
      const uint32_t first = it > (uint32_t)g.stages ? it - (uint32_t)g.stages : 0u;
      for (uint32_t j = first; j < it; ++j)
        if (!tc::mbar_wait(TC_FULL(j % (uint32_t)g.stages), (j / (uint32_t)g.stages) & 1u)) atomicOr(g.err, 2u);
    }
  } else if (w == 1) {
    // ---- MMA issuer ------------------------------------------------------------------
    if (lane == 0) {
      uint32_t it = 0;
      int np = 0;
      bool ok = true;
      const uint32_t sbo = (uint32_t)g.Kp * 16u;
      for (int p = blockIdx.x; ok && p < npairs; p += gridDim.x, ++np) {
        if (np > 0 && !tc::mbar_wait(ACC_EMPTY, (uint32_t)(np - 1) & 1u)) {
          ok = false;
          atomicOr(g.err, 4u);
          break;
        }
        tc::fence_after_sync();
        for (int l = 0; l < 81; ++l, ++it) {
          const int s = (int)(it % (uint32_t)g.stages);
          const uint32_t ph = (it / (uint32_t)g.stages) & 1u;
          if (!tc::mbar_wait(TC_FULL(s), ph)) {
            ok = false;
            atomicOr(g.err, 8u);
            break;
          }
          tc::fence_after_sync();
          const uint32_t abase = ring + (uint32_t)s * stage_bytes;
          const uint32_t bbase = abase + g.sites * g.parts * g.a_sbytes;
          for (int ks = 0; ks < g.Kp / 16; ++ks) {
            const uint64_t bd = tc::smem_desc(bbase + 256u * ks, 128u, sbo);
            for (int p = 0; p < g.parts; ++p) {
              const uint64_t ad =
                  tc::smem_desc(abase + p * g.sites * g.a_sbytes + 2u * g.lbo_a * ks, g.lbo_a, g.sbo_a);
              tc::mma_f16(tmem, ad, bd, g.idesc, (l | ks | p) != 0 ? 1u : 0u);
            }
          }
          tc::mma_commit(TC_EMPTY(s));
        }
        if (ok) tc::mma_commit(ACC_FULL);
      }
      // all MMAs issued by this thread complete before the accumulator is freed
      tc::mma_commit(DRAIN);
      if (!tc::mbar_wait(DRAIN, 0u)) atomicOr(g.err, 16u);
    }
  } else {
    // ---- epilogue: TMEM lane quarter (w % 4) --------------------------------------------
    const int q = w & 3;
    const int row = 32 * q + lane;
    const int si = row / g.MS, mrow = row % g.MS;
    const int j = mrow >> 1, ri = mrow & 1;
    const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(si * g.NS);
    float inv[RMAX];
#pragma unroll
    for (int r = 0; r < RMAX; ++r) inv[r] = r < g.R ? pow2f(-scale_exp(g.xmax[r])) : 0.f;
    int np = 0;
    for (int p = blockIdx.x; p < npairs; p += gridDim.x, ++np) {
      const bool ok = tc::mbar_wait(ACC_FULL, (uint32_t)np & 1u);
      if (!__all_sync(FULL_MASK, ok)) {
        if (lane == 0) atomicOr(g.err, 32u);
        break;
      }
      tc::fence_after_sync();
      float d[4 * TC_RPMAX];
#pragma unroll
      for (int c8 = 0; c8 < TC_RPMAX / 2; ++c8)
        if (8 * c8 < g.NS) tc::tmem_ld8(taddr + 8u * c8, d + 8 * c8);
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(ACC_EMPTY);
      const int site = p * g.sites + si;
      const bool valid = site < g.Vc && j < g.n;
      const float sinv = valid ? pow2f(-__ldg(g.sexp + site)) : 0.f;
#pragma unroll
      for (int r = 0; r < TC_RPMAX; ++r) {
        if (r < g.R) {
          const float P = d[4 * r] + d[4 * r + 2];
          const float Q = d[4 * r + 1] + d[4 * r + 3];
          const float t = __shfl_xor_sync(FULL_MASK, Q, 1);
          float v = (ri ? t + P : P - t) * (inv[r] * sinv);
          if (valid) {
            const size_t e = ((size_t)site * g.n + j) * g.R + r;
            if (g.x) {
              const float xv = reinterpret_cast<const float*>(g.x)[2 * e + ri];
              v += g.shift * xv;
              dot[r] += (double)xv * (double)v;
            }
            reinterpret_cast<float*>(g.y)[2 * e + ri] = v;
          }
        }
      }
    }
  }
#undef TC_FULL
#undef TC_EMPTY
  __syncthreads();
  if (w == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, (uint32_t)g.ncols);
  }
  if (red.result) grid_reduce<RMAX>(dot, red, g.R);
}

// ---------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------

bool coarse_tc_supported(const Coarse& A) {
  return (A.prec == HDCG_F16 || A.prec == HDCG_F32) && A.nvec >= 1 && A.nvec <= 64;
}
static int tc_parts(const Coarse& A) { return A.prec == HDCG_F32 ? 2 : 1; }

void coarse_tc_prepare(Ctx& c, Coarse& A) {
  HDCG_REQUIRE(coarse_tc_supported(A), HDCG_ERR_ARG,
               "tensor-core coarse operator needs an FP16 or FP32 A and Nvec <= 64");
  if (A.tc_ready) return;
  const int parts = tc_parts(A);
  const TcGeom g = tc_geom(A.nvec, 1, parts);
  const size_t nblk = A.Vc * 81;
  A.Atc.ensure(nblk * parts * g.a_gbytes);
  A.sexp.ensure(A.Vc * sizeof(int));
  A.tcs.ensure(sizeof(TcState));
  HDCG_CUDA(cudaMemsetAsync(A.tcs.p, 0, sizeof(TcState), c.stream));
  const size_t nt = nblk * g.rows * g.kgs;
  if (A.prec == HDCG_F32) {
    k_site_scale<float2><<<(unsigned)A.Vc, 256, 0, c.stream>>>(A.A.as<float2>(), A.nvec, A.sexp.as<int>());
    k_a_to_tc<float2><<<(unsigned)((nt + 255) / 256), 256, 0, c.stream>>>(
        A.A.as<float2>(), A.Atc.as<uint4>(), nblk, A.nvec, g.rows, g.kgs, g.a_gbytes, g.lbo_a, g.sbo_a, parts,
        A.sexp.as<int>());
  } else {
    k_site_scale<__half2><<<(unsigned)A.Vc, 256, 0, c.stream>>>(A.A.as<__half2>(), A.nvec, A.sexp.as<int>());
    k_a_to_tc<__half2><<<(unsigned)((nt + 255) / 256), 256, 0, c.stream>>>(
        A.A.as<__half2>(), A.Atc.as<uint4>(), nblk, A.nvec, g.rows, g.kgs, g.a_gbytes, g.lbo_a, g.sbo_a, parts,
        A.sexp.as<int>());
  }
  HDCG_CUDA(cudaGetLastError());
  c.launches += 2;
  A.tc_ready = true;
}

void coarse_tc_check(Ctx& c, Coarse& A) {
  unsigned err = 0;
  HDCG_CUDA(cudaMemcpyAsync(&err, &A.tcs.as<TcState>()->err, sizeof(unsigned), cudaMemcpyDeviceToHost, c.stream));
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
  if (err) {
    HDCG_CUDA(cudaMemsetAsync(A.tcs.p, 0, sizeof(unsigned), c.stream));
    throw Error{HDCG_ERR_TIMEOUT, "tensor-core coarse apply: a pipeline wait expired (flags " +
                                      std::to_string(err) + ")"};
  }
}

void coarse_tc_max(Ctx& c, const float2* x, size_t ne, int R, unsigned* xmax) {
  HDCG_CUDA(cudaMemsetAsync(xmax, 0, RMAX * sizeof(unsigned), c.stream));
  k_cmax<<<(unsigned)((ne + 255) / 256), 256, 0, c.stream>>>(x, ne, R, xmax);
  HDCG_CUDA(cudaGetLastError());
  c.launches += 1;
}

void coarse_tc_to_b(Ctx& c, Coarse& A, int R, const float2* x, const unsigned* xmax, const int* skip) {
  const TcGeom g = tc_geom(A.nvec, R, tc_parts(A));
  A.xtc.ensure(A.Vc * (size_t)g.b_bytes);
  const size_t nt = A.Vc * (size_t)(g.Kp / 8) * g.Rp;
  k_x_to_tc<<<(unsigned)((nt + 255) / 256), 256, 0, c.stream>>>(x, A.xtc.as<uint4>(), A.Vc, A.nvec, R, g.Rp, g.Kp,
                                                                 xmax, skip);
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}

// one launch with cpsm (1 or 2) persistent CTAs per SM and the matching ring
static void launch_tc(Ctx& c, Coarse& A, int R, const float2* x, float2* y, const unsigned* xmax, const int* skip,
                      double* dot_result, double shift, int cpsm) {
  const TcGeom g = tc_geom(A.nvec, R, tc_parts(A), cpsm == 1 ? TC_RING_BYTES_1 : TC_RING_BYTES);
  TcArgs a;
  a.Atc = A.Atc.as<uint4>();
  a.cnbr = A.cnbr.as<int>();
  a.xtc = A.xtc.as<uint4>();
  a.xmax = xmax;
  a.x = x;
  a.y = y;
  a.skip = skip;
  a.err = &A.tcs.as<TcState>()->err;
  a.Vc = (int)A.Vc;
  a.n = A.nvec;
  a.R = R;
  a.sites = g.sites;
  a.MS = g.MS;
  a.Kp = g.Kp;
  a.NS = g.NS;
  a.stages = g.stages;
  a.ncols = g.ncols;
  a.a_gbytes = g.a_gbytes;
  a.a_sbytes = g.a_sbytes;
  a.lbo_a = g.lbo_a;
  a.sbo_a = g.sbo_a;
  a.copy_bytes = g.copy_bytes;
  a.b_bytes = g.b_bytes;
  a.idesc = tc::idesc_f16_f32(128, g.NMMA);
  a.shift = (float)shift;
  a.parts = g.parts;
  a.sexp = A.sexp.as<int>();
  const size_t smem = (size_t)g.stages * g.stage_bytes + (2 * g.stages + 3) * 8 + 16;
  static size_t smem_set = 0;
  if (smem > smem_set) {
    set_smem((const void*)k_capply_tc, std::max<size_t>(smem, 100 * 1024));
    smem_set = std::max<size_t>(smem, 100 * 1024);
  }
  const int npairs = (int)((A.Vc + g.sites - 1) / g.sites);
  const unsigned grid = (unsigned)std::min(npairs, cpsm * device_sms());
  const Reduction red = dot_result ? make_reduction(c, grid, RMAX, dot_result, 0) : Reduction{};
  k_capply_tc<<<grid, TC_THREADS, smem, c.stream>>>(a, red);
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}

// The first apply to R vectors of an operator times two persistent shapes, two
// CTAs per SM with a 96 KB ring and one CTA per SM with a 192 KB ring (twice
// the stages in flight), and keeps the faster.  Both run the same MMAs in the
// same order, so the choice never changes a result.  Inside a stream capture
// the two-CTA shape runs untimed.
void coarse_tc_apply(Ctx& c, Coarse& A, int R, const float2* x, float2* y, const unsigned* xmax, const int* skip,
                     double* dot_result, double shift) {
  int cfg = c.tc_force ? c.tc_force : A.tc_cfg[R];
  if (cfg == 0) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    HDCG_CUDA(cudaStreamIsCapturing(c.stream, &cs));
    if (cs != cudaStreamCaptureStatusNone) {
      cfg = 2;
    } else {
      cudaEvent_t e0, e1;
      HDCG_CUDA(cudaEventCreate(&e0));
      HDCG_CUDA(cudaEventCreate(&e1));
      float best = 1e30f;
      for (int cand : {2, 1}) {
        launch_tc(c, A, R, x, y, xmax, skip, dot_result, shift, cand);
        HDCG_CUDA(cudaEventRecord(e0, c.stream));
        for (int i = 0; i < 3; ++i) launch_tc(c, A, R, x, y, xmax, skip, dot_result, shift, cand);
        HDCG_CUDA(cudaEventRecord(e1, c.stream));
        HDCG_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        HDCG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) {
          best = ms;
          cfg = cand;
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      A.tc_cfg[R] = cfg;
    }
  }
  launch_tc(c, A, R, x, y, xmax, skip, dot_result, shift, cfg);
}

// ---------------------------------------------------------------------------------
// coarse CG for R right-hand sides on the tensor-core operator (vectors FP32 [a][k][r])
// ---------------------------------------------------------------------------------

struct CCtlT {
  double rr[2][RMAX];
  double pAp[RMAX];
  double stop[RMAX];
  int done[RMAX];
  int iter;
  int all_done;
};

__global__ void k_cgt_init(const float2* __restrict__ rhs, float2* x, float2* r, float2* p, size_t ne, int R,
                           unsigned* xmax, Reduction red) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v[RMAX];
  float m[RMAX];
#pragma unroll
  for (int q = 0; q < RMAX; ++q) {
    v[q] = 0.0;
    m[q] = 0.f;
  }
  if (t < ne) {
#pragma unroll
    for (int q = 0; q < RMAX; ++q)
      if (q < R) {
        const float2 b = rhs[t * R + q];
        x[t * R + q] = make_float2(0.f, 0.f);
        r[t * R + q] = b;
        p[t * R + q] = b;
        v[q] = (double)b.x * b.x + (double)b.y * b.y;
        m[q] = fmaxf(fabsf(b.x), fabsf(b.y));
      }
  }
#pragma unroll
  for (int q = 0; q < RMAX; ++q) {
    if (q >= R) break;
    float u = m[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) u = fmaxf(u, __shfl_xor_sync(FULL_MASK, u, o));
    if ((threadIdx.x & 31) == 0 && u > 0.f) atomicMax(xmax + q, __float_as_uint(u));
  }
  grid_reduce<RMAX>(v, red, R);
}

__global__ void k_cgt_start(CCtlT* ctl, int R, double tol, int maxiter) {
  int all = 1;
  for (int q = 0; q < R; ++q) {
    ctl->stop[q] = tol * tol * ctl->rr[0][q];
    ctl->done[q] = (ctl->rr[0][q] == 0.0 || maxiter <= 0) ? 1 : 0;
    all &= ctl->done[q];
  }
  ctl->iter = 0;
  ctl->all_done = all;
}

// x += alpha p, r -= alpha w for the right-hand sides still running; |r|^2; clears xmax
__global__ void k_cgt_update(float2* x, float2* r, const float2* __restrict__ p, const float2* __restrict__ w,
                             size_t ne, int R, const CCtlT* ctl, int par, unsigned* xmax, Reduction red) {
  if (ctl->all_done) return;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0)
    for (int q = 0; q < RMAX; ++q) xmax[q] = 0u;
  double v[RMAX];
#pragma unroll
  for (int q = 0; q < RMAX; ++q) v[q] = 0.0;
  if (t < ne) {
#pragma unroll
    for (int q = 0; q < RMAX; ++q) {
      if (q < R) {
        const size_t e = t * R + q;
        float2 rv = r[e];
        if (!ctl->done[q]) {
          const double pap = ctl->pAp[q];
          const float al = (float)(pap > 0 ? ctl->rr[par][q] / pap : 0.0);
          const float2 pv = p[e], wv = w[e];
          float2 xv = x[e];
          xv.x += al * pv.x;
          xv.y += al * pv.y;
          rv.x -= al * wv.x;
          rv.y -= al * wv.y;
          x[e] = xv;
          r[e] = rv;
        }
        v[q] = (double)rv.x * rv.x + (double)rv.y * rv.y;
      }
    }
  }
  grid_reduce<RMAX>(v, red, R);
}

// p = r + beta p for the right-hand sides still running; max|p| of every right-hand side
__global__ void k_cgt_p(float2* p, const float2* __restrict__ r, size_t ne, int R, const CCtlT* ctl, int par,
                        unsigned* xmax) {
  if (ctl->all_done) return;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  float m[RMAX];
#pragma unroll
  for (int q = 0; q < RMAX; ++q) m[q] = 0.f;
  if (t < ne) {
#pragma unroll
    for (int q = 0; q < RMAX; ++q) {
      if (q < R) {
        const size_t e = t * R + q;
        float2 pv = p[e];
        if (!ctl->done[q]) {
          const double ro = ctl->rr[par][q], rn = ctl->rr[par ^ 1][q];
          const float beta = (float)(ro > 0 ? rn / ro : 0.0);
          const float2 rv = r[e];
          pv.x = rv.x + beta * pv.x;
          pv.y = rv.y + beta * pv.y;
          p[e] = pv;
        }
        m[q] = fmaxf(fabsf(pv.x), fabsf(pv.y));
      }
    }
  }
#pragma unroll
  for (int q = 0; q < RMAX; ++q) {
    if (q >= R) break;
    float u = m[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) u = fmaxf(u, __shfl_xor_sync(FULL_MASK, u, o));
    if ((threadIdx.x & 31) == 0 && u > 0.f) atomicMax(xmax + q, __float_as_uint(u));
  }
}

__global__ void k_cgt_check(CCtlT* ctl, int R, int par, int maxiter) {
  if (ctl->all_done) return;
  const int it = ctl->iter + 1;
  ctl->iter = it;
  int all = 1;
  for (int q = 0; q < R; ++q) {
    const double rn = ctl->rr[par ^ 1][q];
    if (!ctl->done[q] && (rn <= ctl->stop[q] || it >= maxiter || !(rn == rn))) ctl->done[q] = 1;
    all &= ctl->done[q];
  }
  ctl->all_done = all;
}

int coarse_cg_tc(Ctx& c, Coarse& A, int R, const void* rhs, void* sol, double tol, int maxiter, double shift) {
  coarse_tc_prepare(c, A);
  const size_t ne = A.Vc * A.nvec;
  const size_t nc = ne * R;
  A.work.ensure(3 * nc * sizeof(float2));
  A.ctl.ensure(sizeof(CCtlT));
  float2* r = A.work.as<float2>();
  float2* p = r + nc;
  float2* w = p + nc;
  CCtlT* ctl = A.ctl.as<CCtlT>();
  unsigned* xmax = A.tcs.as<TcState>()->xmax;
  const int* skip = &ctl->all_done;
  const unsigned ge = (unsigned)((ne + 255) / 256);
  HDCG_CUDA(cudaMemsetAsync(xmax, 0, RMAX * sizeof(unsigned), c.stream));
  k_cgt_init<<<ge, 256, 0, c.stream>>>((const float2*)rhs, (float2*)sol, r, p, ne, R, xmax,
                                       make_reduction(c, ge, RMAX, &ctl->rr[0][0], 0));
  k_cgt_start<<<1, 1, 0, c.stream>>>(ctl, R, tol, maxiter);
  c.launches += 2;
  auto iteration = [&](int par) {
    coarse_tc_to_b(c, A, R, p, xmax, skip);
    coarse_tc_apply(c, A, R, p, w, xmax, skip, &ctl->pAp[0], shift);
    k_cgt_update<<<ge, 256, 0, c.stream>>>((float2*)sol, r, p, w, ne, R, ctl, par, xmax,
                                           make_reduction(c, ge, RMAX, &ctl->rr[par ^ 1][0], 0));
    k_cgt_p<<<ge, 256, 0, c.stream>>>(p, r, ne, R, ctl, par, xmax);
    k_cgt_check<<<1, 1, 0, c.stream>>>(ctl, R, par, maxiter);
    c.launches += 3;
  };
  // pairs of iterations (parities 0, 1): the first directly, later ones as a replayed graph
  uint64_t shift_bits;
  std::memcpy(&shift_bits, &shift, sizeof(shift_bits));
  const std::vector<uintptr_t> key = {(uintptr_t)A.work.p, (uintptr_t)A.ctl.p, (uintptr_t)sol, (uintptr_t)A.Atc.p,
                                      (uintptr_t)A.xtc.p, (uintptr_t)A.tcs.p, (uintptr_t)c.red_partials.p,
                                      (uintptr_t)c.red_ticket.p, (uintptr_t)R, (uintptr_t)maxiter,
                                      (uintptr_t)shift_bits};
  int queued = 0;
  int batch = std::max(2, A.last_iters);
  CCtlT h{};
  while (true) {
    for (int bq = 0; bq < batch && queued < maxiter; bq += 2, queued += 2) {
      if (queued == 0) {
        iteration(0);
        iteration(1);
      } else {
        run_captured(c, A.graph_cg, key, [&] {
          iteration(0);
          iteration(1);
        });
      }
    }
    HDCG_CUDA(cudaGetLastError());
    HDCG_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(CCtlT), cudaMemcpyDeviceToHost, c.stream));
    coarse_tc_check(c, A);   // synchronises the stream
    if (h.all_done || queued >= maxiter) break;
    batch = 2;
  }
  A.last_iters = std::max(1, h.iter);
  return h.iter;
}

// ---------------------------------------------------------------------------------
// canonical multi-right-hand-side apply: x, y [R][Vc][Nvec] complex double (device)
// ---------------------------------------------------------------------------------

// [r][e] complex double <-> [e][r] complex float or double
template <typename V>
__global__ void k_canon_to_multi(const double2* __restrict__ in, V* out, size_t ne, int R) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ne * R) return;
  const size_t e = t / R;
  const int r = (int)(t % R);
  const double2 v = in[(size_t)r * ne + e];
  out[t] = {(decltype(out[t].x))v.x, (decltype(out[t].y))v.y};
}
template <typename V>
__global__ void k_multi_to_canon(const V* __restrict__ in, double2* out, size_t ne, int R) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ne * R) return;
  const size_t e = t / R;
  const int r = (int)(t % R);
  out[(size_t)r * ne + e] = make_double2((double)in[t].x, (double)in[t].y);
}

void coarse_canon_to_multi(Ctx& c, const void* in64, float2* out, size_t ne, int R) {
  k_canon_to_multi<float2><<<(unsigned)((ne * R + 255) / 256), 256, 0, c.stream>>>((const double2*)in64, out, ne, R);
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}
void coarse_multi_to_canon(Ctx& c, const float2* in, void* out64, size_t ne, int R) {
  k_multi_to_canon<float2><<<(unsigned)((ne * R + 255) / 256), 256, 0, c.stream>>>(in, (double2*)out64, ne, R);
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}

int coarse_solve_canon(Ctx& c, Coarse& A, int R, const void* b64, void* x64, double tol, int maxiter) {
  HDCG_REQUIRE(R >= 1 && R <= RMAX, HDCG_ERR_ARG, "1..16 right-hand sides");
  const size_t ne = A.Vc * A.nvec, nc = ne * R;
  const unsigned gt = (unsigned)((nc + 255) / 256);
  DevMem tmp;
  int it;
  if (A.l2) A.l2->last_broke = 0;
  if (A.vec_prec() == HDCG_F32) {
    tmp.ensure(2 * nc * sizeof(float2));
    float2* bi = tmp.as<float2>();
    float2* xi = bi + nc;
    k_canon_to_multi<float2><<<gt, 256, 0, c.stream>>>((const double2*)b64, bi, ne, R);
    it = coarse_cg_multi(c, A, R, bi, xi, tol, maxiter);
    k_multi_to_canon<float2><<<gt, 256, 0, c.stream>>>(xi, (double2*)x64, ne, R);
    HDCG_REQUIRE(!(A.l2 && A.l2->last_broke), HDCG_ERR_BREAKDOWN,
                 "level-1 solve: (p, A p) <= 0 or a non-finite residual before the tolerance");
  } else {
    tmp.ensure(2 * nc * sizeof(double2));
    double2* bi = tmp.as<double2>();
    double2* xi = bi + nc;
    k_canon_to_multi<double2><<<gt, 256, 0, c.stream>>>((const double2*)b64, bi, ne, R);
    it = coarse_cg_multi(c, A, R, bi, xi, tol, maxiter);
    k_multi_to_canon<double2><<<gt, 256, 0, c.stream>>>(xi, (double2*)x64, ne, R);
  }
  c.launches += 2;
  HDCG_CUDA(cudaGetLastError());
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
  return it;
}

// Mean device time of one tensor-core stencil apply (k_capply_tc alone) to R
// Gaussian coarse vectors: 3 warm-up launches, then reps launches between two
// CUDA events on the handle's stream (the B operand is prepared once).
double coarse_tc_time_us(Ctx& c, Coarse& A, int R, int reps) {
  HDCG_REQUIRE(coarse_tc_supported(A), HDCG_ERR_ARG, "the tensor-core apply needs an FP16 or FP32 A, Nvec <= 64");
  HDCG_REQUIRE(R >= 1 && R <= RMAX && reps >= 1, HDCG_ERR_ARG, "1..16 right-hand sides, reps >= 1");
  coarse_tc_prepare(c, A);
  const size_t ne = A.Vc * A.nvec, nc = ne * R;
  DevMem tmp;
  tmp.ensure(2 * nc * sizeof(float2));
  float2* xi = tmp.as<float2>();
  float2* yi = xi + nc;
  coarse_noise(c, xi, nc, 0x7e57);
  unsigned* xmax = A.tcs.as<TcState>()->xmax;
  coarse_tc_max(c, xi, ne, R, xmax);
  coarse_tc_to_b(c, A, R, xi, xmax, nullptr);
  for (int i = 0; i < 3; ++i) coarse_tc_apply(c, A, R, xi, yi, xmax, nullptr, nullptr, 0.0);
  cudaEvent_t e0, e1;
  HDCG_CUDA(cudaEventCreate(&e0));
  HDCG_CUDA(cudaEventCreate(&e1));
  HDCG_CUDA(cudaEventRecord(e0, c.stream));
  for (int i = 0; i < reps; ++i) coarse_tc_apply(c, A, R, xi, yi, xmax, nullptr, nullptr, 0.0);
  HDCG_CUDA(cudaEventRecord(e1, c.stream));
  HDCG_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  HDCG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  coarse_tc_check(c, A);
  return 1e3 * ms / reps;
}

void coarse_apply_multi_canon(Ctx& c, Coarse& A, int R, const void* x64, void* y64) {
  HDCG_REQUIRE(R >= 1 && R <= RMAX, HDCG_ERR_ARG, "1..16 right-hand sides");
  const size_t ne = A.Vc * A.nvec, nc = ne * R;
  const unsigned gt = (unsigned)((nc + 255) / 256);
  if (coarse_tc_supported(A)) {
    coarse_tc_prepare(c, A);
    DevMem tmp;
    tmp.ensure(2 * nc * sizeof(float2));
    float2* xi = tmp.as<float2>();
    float2* yi = xi + nc;
    k_canon_to_multi<float2><<<gt, 256, 0, c.stream>>>((const double2*)x64, xi, ne, R);
    unsigned* xmax = A.tcs.as<TcState>()->xmax;
    coarse_tc_max(c, xi, ne, R, xmax);
    coarse_tc_to_b(c, A, R, xi, xmax, nullptr);
    coarse_tc_apply(c, A, R, xi, yi, xmax, nullptr, nullptr, 0.0);
    k_multi_to_canon<float2><<<gt, 256, 0, c.stream>>>(yi, (double2*)y64, ne, R);
    c.launches += 2;
    HDCG_CUDA(cudaGetLastError());
    coarse_tc_check(c, A);
    return;
  }
  // FP32 / FP64 operator: the CUDA-core kernel on [a][k][r] complex double
  DevMem tmp;
  tmp.ensure(2 * nc * sizeof(double2));
  double2* xi = tmp.as<double2>();
  double2* yi = xi + nc;
  k_canon_to_multi<double2><<<gt, 256, 0, c.stream>>>((const double2*)x64, xi, ne, R);
  coarse_apply_multi(c, A, R, xi, yi);
  k_multi_to_canon<double2><<<gt, 256, 0, c.stream>>>(yi, (double2*)y64, ne, R);
  c.launches += 2;
  HDCG_CUDA(cudaGetLastError());
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
}

}  // namespace hdcg
