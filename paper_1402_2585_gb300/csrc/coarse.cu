// Blocked deflation subspace and little Dirac operator of the HDCG library
// (Boyle, arXiv 1402.2585, Sec. 2, Sec. 5.1, Sec. 5.1.1).
//
// Blocks are 4D boxes spanning all of the fifth dimension.  Kernels that work
// block by block run one CTA per block and stage tiles of TILE consecutive 5D
// sites of all subspace vectors in shared memory:
//  * block Gram matrices G[b][j][k] = <X_j^b, Y_k^b> (FP32 products over one
//    tile, FP64 accumulation across tiles);
//  * in-place block transforms Phi_k^b <- sum_j Phi_j^b T_b[j][k].
// Block orthonormalisation is two rounds of Cholesky-QR (G = R^dag R in FP64,
// Phi <- Phi R^-1): the Q factor of the block QR with positive diagonal, i.e.
// the result of Gram-Schmidt applied twice, up to rounding.
// The little Dirac operator A[a][l][j][k] = <phi_j^a | H | phi_k^{a+delta_l}>
// is assembled by the Fourier trick of Sec. 5.1.1 and applied as the 81-point
// stencil y_a = sum_l A[a][l] x_{a+delta_l}.
#include <algorithm>
#include <cmath>
#include <complex>
#include <type_traits>
#include <vector>

#include "coarse.cuh"

namespace hdcg {

constexpr int TILE = 16;       // 5D sites per shared-memory tile
constexpr int MAX_NVEC = 64;

// ---------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------
void subspace_init(Ctx& c, Subspace& s, const int block[4], int nvec, int prec) {
  HDCG_REQUIRE(nvec >= 1 && nvec <= MAX_NVEC, HDCG_ERR_ARG, "nvec must be in 1..64");
  HDCG_REQUIRE(prec == HDCG_F64 || prec == HDCG_F32 || prec == HDCG_F16, HDCG_ERR_ARG,
               "subspace precision must be F64, F32 or F16");
  for (int mu = 0; mu < 4; ++mu) {
    HDCG_REQUIRE(block[mu] >= 2 && block[mu] % 2 == 0 && c.dims[mu] % block[mu] == 0, HDCG_ERR_ARG,
                 "block extents must be even and divide the lattice");
    s.block[mu] = block[mu];
    s.cdims[mu] = c.dims[mu] / block[mu];
  }
  s.Vc = (size_t)s.cdims[0] * s.cdims[1] * s.cdims[2] * s.cdims[3];
  s.nvec = nvec;
  s.prec = prec;
  s.spb = block[0] * block[1] * block[2] * block[3] / 2;
  HDCG_REQUIRE(((size_t)s.spb * c.Ls) % TILE == 0, HDCG_ERR_ARG, "block too small");
  std::vector<int> bos(c.n4), bsites(s.Vc * s.spb), fill(s.Vc, 0), bc(s.Vc * 4);
  const int L0 = c.dims[0], L1 = c.dims[1], L2 = c.dims[2];
  for (size_t i = 0; i < c.n4; ++i) {
    const int hx = L0 / 2;
    size_t rest = i / hx;
    const int y = (int)(rest % L1);
    rest /= L1;
    const int z = (int)(rest % L2);
    const int t = (int)(rest / L2);
    const int x = 2 * (int)(i % hx) + ((1 + y + z + t) & 1);   // odd parity
    const int bx = x / block[0], by = y / block[1], bz = z / block[2], bt = t / block[3];
    const size_t b = bx + (size_t)s.cdims[0] * (by + (size_t)s.cdims[1] * (bz + (size_t)s.cdims[2] * bt));
    bos[i] = (int)b;
    HDCG_REQUIRE(fill[b] < s.spb, HDCG_ERR_ARG, "block bookkeeping");
    bsites[b * s.spb + fill[b]++] = (int)i;
  }
  for (size_t b = 0; b < s.Vc; ++b) {
    size_t r = b;
    for (int mu = 0; mu < 4; ++mu) {
      bc[b * 4 + mu] = (int)(r % s.cdims[mu]);
      r /= s.cdims[mu];
    }
  }
  s.block_of_site.ensure(bos.size() * sizeof(int));
  s.block_sites.ensure(bsites.size() * sizeof(int));
  s.block_coords.ensure(bc.size() * sizeof(int));
  HDCG_CUDA(cudaMemcpy(s.block_of_site.p, bos.data(), bos.size() * sizeof(int), cudaMemcpyHostToDevice));
  HDCG_CUDA(cudaMemcpy(s.block_sites.p, bsites.data(), bsites.size() * sizeof(int), cudaMemcpyHostToDevice));
  HDCG_CUDA(cudaMemcpy(s.block_coords.p, bc.data(), bc.size() * sizeof(int), cudaMemcpyHostToDevice));
  s.vecs.ensure((size_t)nvec * s.vec_bytes(c));
}

// ---------------------------------------------------------------------------
// Gaussian noise: splitmix64 (Steele, Lea & Flood 2014) as a counter-based
// generator, Box-Muller on consecutive pairs; complex element e uses outputs
// 2e, 2e+1 (E|z|^2 = 1).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double u01(uint64_t z) {
  return ((double)(z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

template <typename S>
__global__ void k_noise(uint4* vecs, size_t n5, size_t nf, uint64_t seed) {
  using R = typename Store<S>::real;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n5 * nf) return;
  R v[24];
  for (int e = 0; e < 12; ++e) {
    const uint64_t ce = t * 12 + e;
    const double u1 = u01(splitmix64_at(seed, 2 * ce));
    const double u2 = u01(splitmix64_at(seed, 2 * ce + 1));
    const double r = sqrt(-2.0 * log(u1)) * 0.70710678118654752440;
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    v[2 * e] = (R)(r * cs);
    v[2 * e + 1] = (R)(r * sn);
  }
  const size_t f = t / n5, site5 = t % n5;
  store_spinor<S, R>(vecs + f * n5 * Store<S>::chunks, site5, n5, v);
}

// n complex Gaussians (E|z|^2 = 1) in canonical order, element e from outputs 2e, 2e+1
__global__ void k_noise_c(float2* out, size_t n, uint64_t seed) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double u1 = u01(splitmix64_at(seed, 2 * t));
  const double u2 = u01(splitmix64_at(seed, 2 * t + 1));
  const double r = sqrt(-2.0 * log(u1)) * 0.70710678118654752440;
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  out[t] = make_float2((float)(r * cs), (float)(r * sn));
}

void coarse_noise(Ctx& c, float2* out, size_t n, uint64_t seed) {
  k_noise_c<<<(unsigned)((n + 255) / 256), 256, 0, c.stream>>>(out, n, seed);
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}

void subspace_noise(Ctx& c, Subspace& s, uint64_t seed) {
  const size_t n = c.n5 * s.nvec;
  DISPATCH_SUB(s.prec, S, { k_noise<S><<<(unsigned)((n + 255) / 256), 256, 0, c.stream>>>(s.vecs.as<uint4>(), c.n5, s.nvec, seed); });
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}

// ---------------------------------------------------------------------------
// shared-memory tiles of a block
// ---------------------------------------------------------------------------
struct BlockArgs {
  const int* block_sites;
  int spb, Ls, lslog2;
  size_t n5;
};

// site5 of the g-th 5D site of block b (sites ascending, s fastest)
__device__ __forceinline__ size_t block_site5(const BlockArgs& ba, size_t b, int g) {
  const int i = g >> ba.lslog2, s = g & (ba.Ls - 1);
  return (size_t)__ldg(ba.block_sites + b * ba.spb + i) * ba.Ls + s;
}

constexpr int TROW = TILE * 24 + 2;  // padded row (floats or doubles) of one vector's tile

// load rows [0, nv) of vectors (base + k * kstride granules) for tile tile0 of block b
template <typename S, typename Rt>
__device__ void load_tile(Rt* sm, const uint4* base, size_t kstride, int nv, const BlockArgs& ba, size_t b,
                          int tile0) {
  using R = typename Store<S>::real;
  constexpr int C = Store<S>::chunks, P = Store<S>::per_chunk;
  const int total = nv * TILE * C;
  for (int q = threadIdx.x; q < total; q += blockDim.x) {
    const int t = q % TILE;
    const int ch = (q / TILE) % C;
    const int k = q / (C * TILE);
    const size_t site5 = block_site5(ba, b, tile0 + t);
    const uint4 g = __ldg(base + k * kstride + ch * ba.n5 + site5);
    R tmp[P];
    unpack(S{}, g, tmp);
#pragma unroll
    for (int i = 0; i < P; ++i) sm[k * TROW + t * 24 + ch * P + i] = (Rt)tmp[i];
  }
}

template <typename S, typename Rt>
__device__ void store_tile(const Rt* sm, uint4* base, size_t kstride, int nv, const BlockArgs& ba, size_t b,
                           int tile0) {
  using R = typename Store<S>::real;
  constexpr int C = Store<S>::chunks, P = Store<S>::per_chunk;
  const int total = nv * TILE * C;
  for (int q = threadIdx.x; q < total; q += blockDim.x) {
    const int t = q % TILE;
    const int ch = (q / TILE) % C;
    const int k = q / (C * TILE);
    const size_t site5 = block_site5(ba, b, tile0 + t);
    R tmp[P];
#pragma unroll
    for (int i = 0; i < P; ++i) tmp[i] = (R)sm[k * TROW + t * 24 + ch * P + i];
    base[k * kstride + ch * ba.n5 + site5] = pack(S{}, tmp);
  }
}

// G[b] (out + b * ostride) [j][k] = phase_b^* <X_j^b, Y_k^b>,  j < nx, k < ny
struct GramPhase {
  int on;
  int n[4];
  int L[4];
  const int* coords;
};

// SAME: Y is X (self Gram matrix): the tile is staged once.
template <typename Sx, typename Sy, typename Rt, bool SAME = false>
__global__ void __launch_bounds__(256) k_block_gram(const uint4* X, size_t xstride, int nx, const uint4* Y,
                                                    size_t ystride, int ny, BlockArgs ba, double2* out,
                                                    size_t ostride, GramPhase ph) {
  extern __shared__ __align__(16) unsigned char smraw[];
  Rt* xs = reinterpret_cast<Rt*>(smraw);
  Rt* ys = SAME ? xs : xs + (size_t)nx * TROW;
  const size_t b = blockIdx.x;
  const int npairs = nx * ny;
  constexpr int MAXP = (MAX_NVEC * MAX_NVEC + 255) / 256;
  double ar[MAXP], ai[MAXP];
#pragma unroll
  for (int q = 0; q < MAXP; ++q) ar[q] = ai[q] = 0.0;
  const int nsites = ba.spb * ba.Ls;
  for (int tile0 = 0; tile0 < nsites; tile0 += TILE) {
    __syncthreads();
    load_tile<Sx, Rt>(xs, X, xstride, nx, ba, b, tile0);
    if (!SAME) load_tile<Sy, Rt>(ys, Y, ystride, ny, ba, b, tile0);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < MAXP; ++q) {
      const int p = threadIdx.x + q * 256;
      if (p < npairs) {
        const int j = p / ny, k = p % ny;
        const Rt* xr = xs + j * TROW;
        const Rt* yr = ys + k * TROW;
        Rt sr = 0, si = 0;
#pragma unroll 8
        for (int e = 0; e < TILE * 24; e += 2) {
          const Rt a = xr[e], bb = xr[e + 1], cc = yr[e], d = yr[e + 1];
          sr += a * cc + bb * d;
          si += a * d - bb * cc;
        }
        ar[q] += (double)sr;
        ai[q] += (double)si;
      }
    }
  }
  double pr = 1.0, pi = 0.0;
  if (ph.on) {
    double arg = 0.0;
    for (int mu = 0; mu < 4; ++mu) arg += (double)ph.n[mu] * ph.coords[b * 4 + mu] / ph.L[mu];
    sincospi(2.0 * arg, &pi, &pr);
    pi = -pi;  // conjugate phase
  }
#pragma unroll
  for (int q = 0; q < MAXP; ++q) {
    const int p = threadIdx.x + q * 256;
    if (p < npairs) out[b * ostride + p] = make_double2(pr * ar[q] - pi * ai[q], pr * ai[q] + pi * ar[q]);
  }
}

// X_k^b <- sum_{j} X_j^b T_b[j][k]  (T: FP64 complex [Vc][n][n]).  Each tile
// of all n vectors is staged in shared memory, then every thread computes
// whole 16-byte granules of the result and stores them in place.
template <typename S, typename Rt>
__global__ void __launch_bounds__(256) k_block_transform(uint4* X, size_t xstride, int n, BlockArgs ba,
                                                         const double2* T) {
  using R = typename Store<S>::real;
  constexpr int C = Store<S>::chunks, P = Store<S>::per_chunk;
  extern __shared__ __align__(16) unsigned char smraw[];
  Rt* xs = reinterpret_cast<Rt*>(smraw);
  Rt* ts = xs + (size_t)n * TROW;     // n*n complex, [j][k] re, im
  const size_t b = blockIdx.x;
  for (int q = threadIdx.x; q < n * n; q += blockDim.x) {
    const double2 v = T[b * n * n + q];
    ts[2 * q] = (Rt)v.x;
    ts[2 * q + 1] = (Rt)v.y;
  }
  const int nsites = ba.spb * ba.Ls;
  const int units = n * TILE * C;
  for (int tile0 = 0; tile0 < nsites; tile0 += TILE) {
    __syncthreads();
    load_tile<S, Rt>(xs, X, xstride, n, ba, b, tile0);
    __syncthreads();
    for (int u = threadIdx.x; u < units; u += blockDim.x) {
      const int t = u % TILE;
      const int ch = (u / TILE) % C;
      const int k = u / (C * TILE);
      Rt o[P];
#pragma unroll
      for (int i = 0; i < P; ++i) o[i] = 0;
      for (int j = 0; j <= k && j < n; ++j) {
        const Rt tr = ts[2 * (j * n + k)], ti = ts[2 * (j * n + k) + 1];
        const Rt* xr = xs + j * TROW + t * 24 + ch * P;
#pragma unroll
        for (int i = 0; i < P; i += 2) {
          o[i] += xr[i] * tr - xr[i + 1] * ti;
          o[i + 1] += xr[i] * ti + xr[i + 1] * tr;
        }
      }
      R w[P];
#pragma unroll
      for (int i = 0; i < P; ++i) w[i] = (R)o[i];
      X[k * xstride + ch * ba.n5 + block_site5(ba, b, tile0 + t)] = pack(S{}, w);
    }
  }
}

// per block: G = R^dag R (Cholesky, FP64); T = R^-1 (upper triangular)
__global__ void k_cholinv(const double2* G, double2* T, int n, size_t Vc, int* fail) {
  const size_t b = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= Vc) return;
  const double2* g = G + b * n * n;
  double2* t = T + b * n * n;
  // R (upper) is built in t, then inverted in place column by column
  for (int q = 0; q < n * n; ++q) t[q] = make_double2(0, 0);
  // Cholesky into t (upper triangle)
  for (int j = 0; j < n; ++j) {
    double d = g[j * n + j].x;
    for (int i = 0; i < j; ++i) d -= t[i * n + j].x * t[i * n + j].x + t[i * n + j].y * t[i * n + j].y;
    if (!(d > 0.0)) {
      atomicExch(fail, 1);
      d = 1.0;
    }
    const double rjj = sqrt(d);
    t[j * n + j] = make_double2(rjj, 0);
    for (int k = j + 1; k < n; ++k) {
      double sr = g[j * n + k].x, si = g[j * n + k].y;
      for (int i = 0; i < j; ++i) {
        // conj(R[i][j]) * R[i][k]
        const double2 a = t[i * n + j], c = t[i * n + k];
        sr -= a.x * c.x + a.y * c.y;
        si -= a.x * c.y - a.y * c.x;
      }
      t[j * n + k] = make_double2(sr / rjj, si / rjj);
    }
  }
  // invert the upper-triangular R in place: solve R X = I column by column
  for (int k = n - 1; k >= 0; --k) {
    // X[k][k] = 1 / R[k][k]; for i < k: X[i][k] = -(sum_{m=i+1..k} R[i][m] X[m][k]) / R[i][i]
    // store X in the same array; R entries in column k rows < k are read before overwrite
    const double rkk = t[k * n + k].x;
    double2 col[MAX_NVEC];
    for (int i = 0; i < n; ++i) col[i] = make_double2(0, 0);
    col[k] = make_double2(1.0 / rkk, 0);
    for (int i = k - 1; i >= 0; --i) {
      double sr = 0, si = 0;
      for (int m = i + 1; m <= k; ++m) {
        const double2 r = t[i * n + m], x = col[m];
        sr += r.x * x.x - r.y * x.y;
        si += r.x * x.y + r.y * x.x;
      }
      const double rii = t[i * n + i].x;
      col[i] = make_double2(-sr / rii, -si / rii);
    }
    // column k of R is no longer needed by later (smaller k) columns? it is: rows i<k of
    // columns m<=k are used when solving column k' < k only for m <= k' < k. Column k
    // itself is not read again, so it can be overwritten.
    for (int i = 0; i <= k; ++i) t[i * n + k] = col[i];
  }
}

static BlockArgs block_args(const Ctx& c, const Subspace& s) {
  BlockArgs ba;
  ba.block_sites = s.block_sites.as<int>();
  ba.spb = s.spb;
  ba.Ls = c.Ls;
  ba.lslog2 = c.lslog2;
  ba.n5 = c.n5;
  return ba;
}

template <typename Rt>
static size_t tile_smem(int nrows) { return (size_t)nrows * TROW * sizeof(Rt); }

static void set_smem_limit(const void* fn, size_t bytes) {
  if (bytes > 48 * 1024) HDCG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

template <typename Sx, typename Sy, typename Rt>
static void launch_gram_t(Ctx& c, const Subspace& s, const uint4* X, int nx, const uint4* Y, int ny,
                          size_t ystride, double2* out, size_t ostride, GramPhase ph) {
  const size_t sm = tile_smem<Rt>(nx + ny);
  auto fn = k_block_gram<Sx, Sy, Rt>;
  set_smem_limit((const void*)fn, sm);
  const size_t xstride = s.vec_bytes(c) / 16;
  fn<<<(unsigned)s.Vc, 256, sm, c.stream>>>(X, xstride, nx, Y, ystride, ny, block_args(c, s), out, ostride, ph);
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}

// G[b][j][k] = <phi_j, Y_k> over block b; Y: ny fields of precision yprec (stride in granules).
// Tiles are FP64 for an FP64 subspace, FP32 otherwise.
static void block_gram(Ctx& c, const Subspace& s, const uint4* Y, int ny, int yprec, size_t ystride,
                       double2* out, size_t ostride, GramPhase ph) {
  DISPATCH_SUB(s.prec, Sx, {
    DISPATCH_PREC(yprec, Sy, {
      using Rt = typename std::conditional<std::is_same<Sx, f64_t>::value, double, float>::type;
      launch_gram_t<Sx, Sy, Rt>(c, s, s.vecs.as<uint4>(), s.nvec, Y, ny, ystride, out, ostride, ph);
    });
  });
}

// self Gram matrix of the subspace blocks with FP64 products (orthonormalisation)
static void block_self_gram(Ctx& c, const Subspace& s, double2* out) {
  const int n = s.nvec;
  const size_t stride = s.vec_bytes(c) / 16;
  const size_t sm = tile_smem<double>(n);
  DISPATCH_SUB(s.prec, Sx, {
    auto fn = k_block_gram<Sx, Sx, double, true>;
    set_smem_limit((const void*)fn, sm);
    fn<<<(unsigned)s.Vc, 256, sm, c.stream>>>(s.vecs.as<uint4>(), stride, n, s.vecs.as<uint4>(), stride, n,
                                               block_args(c, s), out, (size_t)n * n, GramPhase{});
  });
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}

void block_orthonormalise(Ctx& c, Subspace& s) {
  const int n = s.nvec;
  DevMem G, T, fail;
  G.ensure(s.Vc * n * n * sizeof(double2));
  T.ensure(s.Vc * n * n * sizeof(double2));
  fail.ensure(sizeof(int));
  HDCG_CUDA(cudaMemsetAsync(fail.p, 0, sizeof(int), c.stream));
  const size_t stride = s.vec_bytes(c) / 16;
  for (int round = 0; round < 2; ++round) {
    block_self_gram(c, s, G.as<double2>());
    k_cholinv<<<(unsigned)((s.Vc + 63) / 64), 64, 0, c.stream>>>(G.as<double2>(), T.as<double2>(), n, s.Vc,
                                                                  fail.as<int>());
    HDCG_CUDA(cudaGetLastError());
    ++c.launches;
    DISPATCH_SUB(s.prec, S, {
      using Rt = typename std::conditional<std::is_same<S, f64_t>::value, double, float>::type;
      const size_t sm = tile_smem<Rt>(n) + (size_t)n * n * 2 * sizeof(Rt);
      auto fn = k_block_transform<S, Rt>;
      set_smem_limit((const void*)fn, sm);
      fn<<<(unsigned)s.Vc, 256, sm, c.stream>>>(s.vecs.as<uint4>(), stride, n, block_args(c, s), T.as<double2>());
    });
    HDCG_CUDA(cudaGetLastError());
    ++c.launches;
  }
  int h_fail = 0;
  HDCG_CUDA(cudaMemcpyAsync(&h_fail, fail.p, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
  HDCG_REQUIRE(!h_fail, HDCG_ERR_BREAKDOWN, "block Gram matrix not positive definite (rank-deficient subspace)");
}

// ---------------------------------------------------------------------------
// restriction / prolongation
// ---------------------------------------------------------------------------
template <typename C> struct CV;
template <> struct CV<float> { using T = float2; };
template <> struct CV<double> { using T = double2; };

constexpr int RKC = 16;  // subspace vectors per restriction pass

template <typename Sp, typename Sv, typename Rc>
__global__ void __launch_bounds__(256) k_restrict(const uint4* __restrict__ phi, size_t pstride, int nvec,
                                                  const uint4* __restrict__ v, BlockArgs ba,
                                                  typename CV<Rc>::T* out) {
  using Rp = typename Store<Sp>::real;
  using Rv = typename Store<Sv>::real;
  using R = typename std::conditional<(sizeof(Rp) > sizeof(Rv)), Rp, Rv>::type;
  const size_t b = blockIdx.x;
  const int nsites = ba.spb * ba.Ls;
  for (int k0 = 0; k0 < nvec; k0 += RKC) {
    const int kc = min(RKC, nvec - k0);
    R accr[2 * RKC];
#pragma unroll
    for (int q = 0; q < 2 * RKC; ++q) accr[q] = 0;
    for (int g = threadIdx.x; g < nsites; g += blockDim.x) {
      const size_t site5 = block_site5(ba, b, g);
      Rv vv[24];
      load_spinor<Sv, Rv>(v, site5, ba.n5, vv);
#pragma unroll
      for (int q = 0; q < RKC; ++q) {
        if (q < kc) {
          Rp pv[24];
          load_spinor<Sp, Rp>(phi + (size_t)(k0 + q) * pstride, site5, ba.n5, pv);
          R sr = 0, si = 0;
#pragma unroll
          for (int e = 0; e < 24; e += 2) {
            sr += (R)pv[e] * (R)vv[e] + (R)pv[e + 1] * (R)vv[e + 1];
            si += (R)pv[e] * (R)vv[e + 1] - (R)pv[e + 1] * (R)vv[e];
          }
          accr[2 * q] += sr;
          accr[2 * q + 1] += si;
        }
      }
    }
    double acc[2 * RKC];
#pragma unroll
    for (int q = 0; q < 2 * RKC; ++q) acc[q] = (double)accr[q];
    block_sum<2 * RKC>(acc);
    if (threadIdx.x == 0)
      for (int q = 0; q < kc; ++q) out[b * nvec + k0 + q] = {(Rc)acc[2 * q], (Rc)acc[2 * q + 1]};
    __syncthreads();
  }
}

void restrict_field(Ctx& c, const Subspace& s, const uint4* v, int vprec, void* cvec, int cprec) {
  const size_t pstride = s.vec_bytes(c) / 16;
  HDCG_REQUIRE((cprec == HDCG_F64) == (s.prec == HDCG_F64), HDCG_ERR_ARG,
               "coarse vectors are FP64 exactly when the subspace is FP64");
  DISPATCH_SUB(s.prec, Sp, {
    DISPATCH_PREC(vprec, Sv, {
      using Rc = typename std::conditional<std::is_same<Sp, f64_t>::value, double, float>::type;
      k_restrict<Sp, Sv, Rc><<<(unsigned)s.Vc, 256, 0, c.stream>>>(s.vecs.as<uint4>(), pstride, s.nvec, v,
                                                                   block_args(c, s), (typename CV<Rc>::T*)cvec);
    });
  });
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}

template <typename Sp, typename So, typename Rc>
__global__ void __launch_bounds__(256) k_prolong(const uint4* __restrict__ phi, size_t pstride, int nvec,
                                                 const typename CV<Rc>::T* __restrict__ cv,
                                                 const int* __restrict__ bos, size_t n5, int lslog2,
                                                 const uint4* add, uint4* out) {
  using Rp = typename Store<Sp>::real;
  using Ro = typename Store<So>::real;
  using R = typename std::conditional<(sizeof(Rp) > sizeof(Ro)), Rp, Ro>::type;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n5) return;
  const int b = __ldg(bos + (t >> lslog2));
  R acc[24];
  if (add) {
    Ro a[24];
    load_spinor<So, Ro>(add, t, n5, a);
#pragma unroll
    for (int e = 0; e < 24; ++e) acc[e] = (R)a[e];
  } else {
#pragma unroll
    for (int e = 0; e < 24; ++e) acc[e] = 0;
  }
  for (int k = 0; k < nvec; ++k) {
    const typename CV<Rc>::T ck = cv[(size_t)b * nvec + k];
    const R cr = (R)ck.x, ci = (R)ck.y;
    Rp pv[24];
    load_spinor<Sp, Rp>(phi + (size_t)k * pstride, t, n5, pv);
#pragma unroll
    for (int e = 0; e < 24; e += 2) {
      acc[e] += cr * (R)pv[e] - ci * (R)pv[e + 1];
      acc[e + 1] += cr * (R)pv[e + 1] + ci * (R)pv[e];
    }
  }
  Ro o[24];
#pragma unroll
  for (int e = 0; e < 24; ++e) o[e] = (Ro)acc[e];
  store_spinor<So, Ro>(out, t, n5, o);
}

void prolong_field(Ctx& c, const Subspace& s, const void* cvec, int cprec, uint4* out, int oprec,
                   const uint4* add) {
  const size_t pstride = s.vec_bytes(c) / 16;
  const unsigned g = (unsigned)((c.n5 + 255) / 256);
  HDCG_REQUIRE((cprec == HDCG_F64) == (s.prec == HDCG_F64), HDCG_ERR_ARG,
               "coarse vectors are FP64 exactly when the subspace is FP64");
  DISPATCH_SUB(s.prec, Sp, {
    DISPATCH_PREC(oprec, So, {
      using Rc = typename std::conditional<std::is_same<Sp, f64_t>::value, double, float>::type;
      k_prolong<Sp, So, Rc><<<g, 256, 0, c.stream>>>(s.vecs.as<uint4>(), pstride, s.nvec,
                                                     (const typename CV<Rc>::T*)cvec, s.block_of_site.as<int>(),
                                                     c.n5, c.lslog2, add, out);
    });
  });
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}

// ---------------------------------------------------------------------------
// little Dirac operator: assembly (Fourier trick) and 81-point apply
// ---------------------------------------------------------------------------
static void offsets_of(int l, int d[4]) {
  for (int mu = 0; mu < 4; ++mu) {
    d[mu] = l % 3 - 1;
    l /= 3;
  }
}

// distinct offsets stored along a dimension of coarse extent L (see hdcg.h)
static std::vector<int> kept_offsets(int L) {
  if (L >= 3) return {-1, 0, 1};
  if (L == 2) return {0, 1};
  return {0};
}
static std::vector<int> momenta_of(int L) {
  if (L >= 3) return {-1, 0, 1};
  std::vector<int> m;
  for (int n = 0; n < L; ++n) m.push_back(n);
  return m;
}

void coarse_init(Ctx& c, Coarse& A, const Subspace& s, int prec) {
  HDCG_REQUIRE(prec == HDCG_F64 || prec == HDCG_F32 || prec == HDCG_F16, HDCG_ERR_ARG,
               "coarse precision must be F64, F32 or F16");
  A.prec = prec;
  A.tc_ready = false;
  A.tc_choice = -1;
  for (int& v : A.tc_cfg) v = 0;
  A.defl.nd = 0;            // a deflation space belongs to the operator it was built for
  A.defl.lam_h.clear();
  A.graph_cg.reset();
  A.graph_ad1.reset();
  A.Aacc.release();
  A.qt.order = 0;           // the preconditioner belongs to the operator it was built from
  // a level-2 subspace of the same geometry is kept (subspace reuse); its
  // operator belongs to the old A and is rebuilt with hdcg_build_coarse(level 2)
  if (A.l2 && (A.l2->Vc1 != s.Vc || A.l2->n1 != s.nvec)) {
    delete A.l2;
    A.l2 = nullptr;
  }
  if (A.l2) {
    A.l2->have_A2 = false;
    A.l2->graph.reset();
  }
  A.nvec = s.nvec;
  A.Vc = s.Vc;
  std::vector<int> nb(s.Vc * 81);
  for (size_t a = 0; a < s.Vc; ++a) {
    int x[4];
    size_t r = a;
    for (int mu = 0; mu < 4; ++mu) {
      x[mu] = (int)(r % s.cdims[mu]);
      r /= s.cdims[mu];
    }
    for (int l = 0; l < 81; ++l) {
      int d[4];
      offsets_of(l, d);
      size_t idx = 0, mul = 1;
      for (int mu = 0; mu < 4; ++mu) {
        const int y = ((x[mu] + d[mu]) % s.cdims[mu] + s.cdims[mu]) % s.cdims[mu];
        idx += y * mul;
        mul *= s.cdims[mu];
      }
      nb[a * 81 + l] = (int)idx;
    }
  }
  A.cnbr.ensure(nb.size() * sizeof(int));
  HDCG_CUDA(cudaMemcpy(A.cnbr.p, nb.data(), nb.size() * sizeof(int), cudaMemcpyHostToDevice));
  const size_t esz = prec == HDCG_F64 ? 16 : prec == HDCG_F32 ? 8 : 4;
  A.A.ensure(s.Vc * 81 * s.nvec * s.nvec * esz);
}

// out = phi_k * exp(i 2 pi n . x_b / L) in precision So
template <typename Sp, typename So>
__global__ void k_phase(const uint4* __restrict__ phi, uint4* out, size_t n5, int lslog2, const int* bos,
                        const int* coords, int4 n, int4 L) {
  using Rp = typename Store<Sp>::real;
  using Ro = typename Store<So>::real;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n5) return;
  const int b = bos[t >> lslog2];
  const int* x = coords + b * 4;
  // exact rational argument: sum n_mu x_mu / L_mu, reduced mod 1 before the sine
  const double arg = (double)n.x * x[0] / L.x + (double)n.y * x[1] / L.y + (double)n.z * x[2] / L.z +
                     (double)n.w * x[3] / L.w;
  double sn, cs;
  if (sizeof(Ro) == 8) {
    sincospi(2.0 * arg, &sn, &cs);
  } else {
    float fs, fc;
    sincospif((float)(2.0 * (arg - floor(arg))), &fs, &fc);
    sn = fs;
    cs = fc;
  }
  Rp v[24];
  load_spinor<Sp, Rp>(phi, t, n5, v);
  Ro o[24];
  const Ro pr = (Ro)cs, pi = (Ro)sn;
#pragma unroll
  for (int e = 0; e < 24; e += 2) {
    o[e] = pr * (Ro)v[e] - pi * (Ro)v[e + 1];
    o[e + 1] = pr * (Ro)v[e + 1] + pi * (Ro)v[e];
  }
  store_spinor<So, Ro>(out, t, n5, o);
}

// A[a][l][k][j] = sum_s Minv[q(l)][s] F[a][s][j][k] for stored l (q(l) >= 0), 0 otherwise
template <typename AT>
__global__ void k_fourier_solve(const double2* __restrict__ F, const double2* __restrict__ Minv,
                                const int* __restrict__ lq, int nS, int n, size_t Vc, AT* A) {
  using R = typename std::conditional<sizeof(AT) == 16, double, float>::type;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t per = (size_t)81 * n * n;
  if (t >= Vc * per) return;
  const size_t a = t / per;
  const int rem = (int)(t % per);
  const int l = rem / (n * n);
  const int k = (rem / n) % n;
  const int j = rem % n;
  const int q = lq[l];
  R sr = 0, si = 0;
  if (q >= 0) {
    for (int s = 0; s < nS; ++s) {
      const double2 m = Minv[q * nS + s];
      const double2 f = F[(a * nS + s) * n * n + j * n + k];
      const R mr = (R)m.x, mi = (R)m.y, fr = (R)f.x, fi = (R)f.y;
      sr += mr * fr - mi * fi;
      si += mr * fi + mi * fr;
    }
  }
  const size_t o = ((a * 81 + l) * n + k) * n + j;
  if constexpr (sizeof(AT) == 16) A[o] = make_double2(sr, si);
  else if constexpr (sizeof(AT) == 8) ((float2*)A)[o] = make_float2((float)sr, (float)si);
  else ((__half2*)A)[o] = __floats2half2_rn((float)sr, (float)si);
}

void coarse_assemble(Ctx& c, Coarse& A, const Subspace& s, int hprec) {
  A.tc_ready = false;
  A.tc_choice = -1;
  for (int& v : A.tc_cfg) v = 0;
  const int n = s.nvec;
  // per-dimension offsets and momenta; compact index q = qx + nx (qy + ny (qz + nz qt))
  std::vector<int> offs[4], moms[4];
  int cnt[4];
  for (int mu = 0; mu < 4; ++mu) {
    offs[mu] = kept_offsets(s.cdims[mu]);
    moms[mu] = momenta_of(s.cdims[mu]);
    cnt[mu] = (int)offs[mu].size();
  }
  const int nS = cnt[0] * cnt[1] * cnt[2] * cnt[3];
  // Minv = kron of per-dimension inverses of M_mu[n][delta] = exp(i 2 pi n delta / L_mu)
  std::vector<std::vector<std::complex<double>>> inv(4);
  for (int mu = 0; mu < 4; ++mu) {
    const int m = cnt[mu];
    std::vector<std::complex<double>> M(m * m), I(m * m);
    for (int a = 0; a < m; ++a)
      for (int d = 0; d < m; ++d)
        M[a * m + d] = std::polar(1.0, 2 * M_PI * moms[mu][a] * offs[mu][d] / (double)s.cdims[mu]);
    // Gauss-Jordan inverse (m <= 3)
    for (int a = 0; a < m; ++a)
      for (int d = 0; d < m; ++d) I[a * m + d] = (a == d) ? 1.0 : 0.0;
    for (int col = 0; col < m; ++col) {
      int piv = col;
      for (int r = col + 1; r < m; ++r)
        if (std::abs(M[r * m + col]) > std::abs(M[piv * m + col])) piv = r;
      for (int k = 0; k < m; ++k) {
        std::swap(M[col * m + k], M[piv * m + k]);
        std::swap(I[col * m + k], I[piv * m + k]);
      }
      const std::complex<double> p = M[col * m + col];
      for (int k = 0; k < m; ++k) {
        M[col * m + k] /= p;
        I[col * m + k] /= p;
      }
      for (int r = 0; r < m; ++r)
        if (r != col) {
          const std::complex<double> f = M[r * m + col];
          for (int k = 0; k < m; ++k) {
            M[r * m + k] -= f * M[col * m + k];
            I[r * m + k] -= f * I[col * m + k];
          }
        }
    }
    inv[mu] = I;  // inv[mu][delta][n]  (inverse of M[n][delta] indexes [delta][n])
  }
  std::vector<double2> Minv((size_t)nS * nS);
  for (int ql = 0; ql < nS; ++ql)
    for (int qs = 0; qs < nS; ++qs) {
      std::complex<double> v = 1.0;
      int rl = ql, rs = qs;
      for (int mu = 0; mu < 4; ++mu) {
        const int il = rl % cnt[mu], is = rs % cnt[mu];
        rl /= cnt[mu];
        rs /= cnt[mu];
        v *= inv[mu][il * cnt[mu] + is];
      }
      Minv[(size_t)ql * nS + qs] = make_double2(v.real(), v.imag());
    }
  // stencil index l -> compact offset index q (or -1)
  std::vector<int> lq(81, -1);
  for (int l = 0; l < 81; ++l) {
    int d[4];
    offsets_of(l, d);
    int q = 0, mul = 1;
    bool ok = true;
    for (int mu = 0; mu < 4; ++mu) {
      int pos = -1;
      for (int i = 0; i < cnt[mu]; ++i)
        if (offs[mu][i] == d[mu]) pos = i;
      if (pos < 0) ok = false;
      q += pos * mul;
      mul *= cnt[mu];
    }
    lq[l] = ok ? q : -1;
  }
  DevMem dMinv, dlq, F, W;
  dMinv.ensure(Minv.size() * sizeof(double2));
  dlq.ensure(81 * sizeof(int));
  HDCG_CUDA(cudaMemcpy(dMinv.p, Minv.data(), Minv.size() * sizeof(double2), cudaMemcpyHostToDevice));
  HDCG_CUDA(cudaMemcpy(dlq.p, lq.data(), 81 * sizeof(int), cudaMemcpyHostToDevice));
  F.ensure(s.Vc * nS * n * n * sizeof(double2));
  W.ensure((size_t)n * c.field_bytes(hprec));
  uint4* ph = c.scratch(hprec, 2);
  const size_t wstride = c.field_bytes(hprec) / 16;
  const unsigned g5 = (unsigned)((c.n5 + 255) / 256);
  for (int qs = 0; qs < nS; ++qs) {
    int mom[4];
    int r = qs;
    for (int mu = 0; mu < 4; ++mu) {
      mom[mu] = moms[mu][r % cnt[mu]];
      r /= cnt[mu];
    }
    for (int k = 0; k < n; ++k) {
      DISPATCH_SUB(s.prec, Sp, {
        DISPATCH_HI(hprec, So, {
          k_phase<Sp, So><<<g5, 256, 0, c.stream>>>(s.vec(c, k), ph, c.n5, c.lslog2, s.block_of_site.as<int>(),
                                                    s.block_coords.as<int>(), make_int4(mom[0], mom[1], mom[2], mom[3]),
                                                    make_int4(s.cdims[0], s.cdims[1], s.cdims[2], s.cdims[3]));
        });
      });
      HDCG_CUDA(cudaGetLastError());
      ++c.launches;
      apply_mdagm(c, hprec, ph, W.as<uint4>() + (size_t)k * wstride, nullptr);
    }
    GramPhase gp;
    gp.on = 1;
    for (int mu = 0; mu < 4; ++mu) {
      gp.n[mu] = mom[mu];
      gp.L[mu] = s.cdims[mu];
    }
    gp.coords = s.block_coords.as<int>();
    block_gram(c, s, W.as<uint4>(), n, hprec, wstride, F.as<double2>() + (size_t)qs * n * n, (size_t)nS * n * n, gp);
  }
  const size_t tot = s.Vc * 81 * n * n;
  const unsigned gA = (unsigned)((tot + 255) / 256);
  if (A.prec == HDCG_F64)
    k_fourier_solve<double2><<<gA, 256, 0, c.stream>>>(F.as<double2>(), dMinv.as<double2>(), dlq.as<int>(), nS, n, s.Vc,
                                                       A.A.as<double2>());
  else if (A.prec == HDCG_F32)
    k_fourier_solve<float2><<<gA, 256, 0, c.stream>>>(F.as<double2>(), dMinv.as<double2>(), dlq.as<int>(), nS, n, s.Vc,
                                                      A.A.as<float2>());
  else {
    k_fourier_solve<__half2><<<gA, 256, 0, c.stream>>>(F.as<double2>(), dMinv.as<double2>(), dlq.as<int>(), nS, n, s.Vc,
                                                       A.A.as<__half2>());
    A.Aacc.ensure(tot * sizeof(float2));
    k_fourier_solve<float2><<<gA, 256, 0, c.stream>>>(F.as<double2>(), dMinv.as<double2>(), dlq.as<int>(), nS, n, s.Vc,
                                                      A.Aacc.as<float2>());
    ++c.launches;
  }
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
}

// y[a][j] = sum_l sum_k A[a][l][k][j] x[a + l][k].  The 81 couplings of a coarse
// site are split over CGROUPS CTAs; CTA (a, g) writes its partial sum to
// y_part[g][a][j] (consumers add the CGROUPS partials).  Within a CTA each warp
// takes one coupling block at a time, lanes run over j (coalesced reads of the
// transposed block A[a][l][k][:]) and the k loop is unrolled so that several
// loads are in flight per lane.
constexpr int CGROUPS = 3;
constexpr int CWARPS = 8;
template <typename AT> constexpr int vec_width() { return 16 / (int)sizeof(AT); }

template <typename AT, typename R>
__device__ __forceinline__ void ld_a(const AT* p, R& re, R& im);
template <> __device__ __forceinline__ void ld_a<double2, double>(const double2* p, double& re, double& im) {
  const double2 v = __ldg(p);
  re = v.x;
  im = v.y;
}
template <> __device__ __forceinline__ void ld_a<float2, float>(const float2* p, float& re, float& im) {
  const float2 v = __ldg(p);
  re = v.x;
  im = v.y;
}
template <> __device__ __forceinline__ void ld_a<__half2, float>(const __half2* p, float& re, float& im) {
  const float2 v = __half22float2(__ldg(p));
  re = v.x;
  im = v.y;
}

// 16-byte vector of VJ consecutive complex entries of A (VJ = 16 / sizeof(AT))
template <typename AT, typename R, int VJ>
__device__ __forceinline__ void ld_a_vec(const AT* p, R* re, R* im) {
  if constexpr (VJ == 1) {
    ld_a<AT, R>(p, re[0], im[0]);
  } else if constexpr (sizeof(AT) == 8) {  // float2 x 2
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    re[0] = v.x; im[0] = v.y; re[1] = v.z; im[1] = v.w;
  } else {  // half2 x 4
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
    float2 f;
    f = h2f(v.x); re[0] = f.x; im[0] = f.y;
    f = h2f(v.y); re[1] = f.x; im[1] = f.y;
    f = h2f(v.z); re[2] = f.x; im[2] = f.y;
    f = h2f(v.w); re[3] = f.x; im[3] = f.y;
  }
}

// Warp layout: lane = ks * NJ + jp with NJ = n / VJ column groups (jp) and
// KS = 32 / NJ row subgroups (ks); a lane reads VJ consecutive j of rows
// k = ks, ks + KS, ... with one 16-byte load per row (for NJ > 32 a lane
// also takes column group jp + 32).  Row partial sums are combined across
// the KS subgroups with shuffles, then across warps in shared memory.
template <typename AT, typename R, int VJ>
__device__ __forceinline__ void capply_body(const AT* __restrict__ A, const int* __restrict__ cnbr, int n,
                                            const typename CV<R>::T* __restrict__ x, typename CV<R>::T* ypart,
                                            size_t nc, double* dot_out) {
  __shared__ double sre[CWARPS][64], sim[CWARPS][64];
  const size_t a = blockIdx.x / CGROUPS;
  const int g = blockIdx.x % CGROUPS;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int NJ = n / VJ;
  const int KS = NJ <= 32 ? 32 / NJ : 1;
  const int ks = NJ <= 32 ? lane / NJ : 0;
  const int jp0 = NJ <= 32 ? lane % NJ : lane;
  const bool on0 = ks < KS && jp0 < NJ;
  const bool on1 = NJ > 32 && lane + 32 < NJ;
  const int l0 = g * 27, l1 = l0 + 27;
  R sr[2 * VJ], si[2 * VJ];
#pragma unroll
  for (int q = 0; q < 2 * VJ; ++q) sr[q] = si[q] = 0;
  for (int l = l0 + w; l < l1; l += CWARPS) {
    const int nb = __ldg(cnbr + a * 81 + l);
    const AT* blk = A + ((a * 81 + l) * n) * n;
    const typename CV<R>::T* xv = x + (size_t)nb * n;
    int k = ks;
    for (; k + 3 * KS < n; k += 4 * KS) {
      R ar[4][2 * VJ], ai[4][2 * VJ];
      typename CV<R>::T xk[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        xk[u] = xv[k + u * KS];
#pragma unroll
        for (int q = 0; q < 2 * VJ; ++q) ar[u][q] = ai[u][q] = 0;
        if (on0) ld_a_vec<AT, R, VJ>(blk + (size_t)(k + u * KS) * n + jp0 * VJ, ar[u], ai[u]);
        if (on1) ld_a_vec<AT, R, VJ>(blk + (size_t)(k + u * KS) * n + (jp0 + 32) * VJ, ar[u] + VJ, ai[u] + VJ);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int q = 0; q < 2 * VJ; ++q) {
          sr[q] += ar[u][q] * xk[u].x - ai[u][q] * xk[u].y;
          si[q] += ar[u][q] * xk[u].y + ai[u][q] * xk[u].x;
        }
    }
    for (; k < n; k += KS) {
      const typename CV<R>::T xk = xv[k];
      R ar[2 * VJ], ai[2 * VJ];
#pragma unroll
      for (int q = 0; q < 2 * VJ; ++q) ar[q] = ai[q] = 0;
      if (on0) ld_a_vec<AT, R, VJ>(blk + (size_t)k * n + jp0 * VJ, ar, ai);
      if (on1) ld_a_vec<AT, R, VJ>(blk + (size_t)k * n + (jp0 + 32) * VJ, ar + VJ, ai + VJ);
#pragma unroll
      for (int q = 0; q < 2 * VJ; ++q) {
        sr[q] += ar[q] * xk.x - ai[q] * xk.y;
        si[q] += ar[q] * xk.y + ai[q] * xk.x;
      }
    }
  }
  // combine the KS row subgroups: lanes ks * NJ + jp (same jp) hold partials of the same j
  if (NJ <= 32) {
    for (int d = 1; d < KS; d <<= 1) {
#pragma unroll
      for (int q = 0; q < VJ; ++q) {
        const R tr = __shfl_down_sync(FULL_MASK, sr[q], d * NJ);
        const R ti = __shfl_down_sync(FULL_MASK, si[q], d * NJ);
        if ((ks & (2 * d - 1)) == 0 && ks + d < KS) {
          sr[q] += tr;
          si[q] += ti;
        }
      }
    }
  }
  if (ks == 0 && jp0 < NJ) {
#pragma unroll
    for (int q = 0; q < VJ; ++q) {
      sre[w][jp0 * VJ + q] = (double)sr[q];
      sim[w][jp0 * VJ + q] = (double)si[q];
    }
  }
  if (on1) {
#pragma unroll
    for (int q = 0; q < VJ; ++q) {
      sre[w][(jp0 + 32) * VJ + q] = (double)sr[VJ + q];
      sim[w][(jp0 + 32) * VJ + q] = (double)si[VJ + q];
    }
  }
  __syncthreads();
  double dv = 0.0;
  if (threadIdx.x < n) {
    double tr = 0, ti = 0;
#pragma unroll
    for (int q = 0; q < CWARPS; ++q) {
      tr += sre[q][threadIdx.x];
      ti += sim[q][threadIdx.x];
    }
    ypart[g * nc + a * n + threadIdx.x] = {(R)tr, (R)ti};
    const typename CV<R>::T xa = x[a * n + threadIdx.x];
    dv = (double)xa.x * tr + (double)xa.y * ti;   // Re conj(x) y (partial over this group)
  }
  *dot_out = dv;
}

template <typename AT, typename R, int VJ>
__global__ void __launch_bounds__(256) k_coarse_apply(const AT* __restrict__ A, const int* __restrict__ cnbr,
                                                      int n, const typename CV<R>::T* __restrict__ x,
                                                      typename CV<R>::T* ypart, size_t nc, int do_red,
                                                      Reduction red) {
  double dv = 0.0;
  capply_body<AT, R, VJ>(A, cnbr, n, x, ypart, nc, &dv);
  double v[1] = {dv};
  if (do_red) grid_reduce<1>(v, red);
}

// y = sum of the CGROUPS partials
template <typename R>
__global__ void k_sum_groups(const typename CV<R>::T* ypart, typename CV<R>::T* y, size_t nc) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nc) return;
  typename CV<R>::T v = ypart[t];
#pragma unroll
  for (int g = 1; g < CGROUPS; ++g) {
    const typename CV<R>::T u = ypart[g * nc + t];
    v.x += u.x;
    v.y += u.y;
  }
  y[t] = v;
}

template <typename AT, typename R>
static void coarse_apply_t(Ctx& c, const Coarse& A, const void* x, void* y, double* xAx) {
  using V = typename CV<R>::T;
  const size_t nc = A.Vc * A.nvec;
  DevMem part;
  part.ensure(CGROUPS * nc * sizeof(V));
  const unsigned g = (unsigned)(A.Vc * CGROUPS);
  Reduction red{};
  if (xAx) red = make_reduction(c, g, 1, xAx, 0);
  if (A.nvec % vec_width<AT>() == 0)
    k_coarse_apply<AT, R, vec_width<AT>()><<<g, 256, 0, c.stream>>>(A.A.as<AT>(), A.cnbr.as<int>(), A.nvec,
                                                                     (const V*)x, part.as<V>(), nc, xAx != nullptr, red);
  else
    k_coarse_apply<AT, R, 1><<<g, 256, 0, c.stream>>>(A.A.as<AT>(), A.cnbr.as<int>(), A.nvec, (const V*)x,
                                                      part.as<V>(), nc, xAx != nullptr, red);
  k_sum_groups<R><<<(unsigned)((nc + 255) / 256), 256, 0, c.stream>>>(part.as<V>(), (V*)y, nc);
  HDCG_CUDA(cudaGetLastError());
  c.launches += 2;
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
}

void coarse_apply(Ctx& c, const Coarse& A, const void* x, void* y, double* xAx) {
  HDCG_REQUIRE(A.nvec <= 64, HDCG_ERR_ARG, "nvec <= 64");
  if (A.prec == HDCG_F64) coarse_apply_t<double2, double>(c, A, x, y, xAx);
  else if (A.prec == HDCG_F32) coarse_apply_t<float2, float>(c, A, x, y, xAx);
  else coarse_apply_t<__half2, float>(c, A, x, y, xAx);
}

// ---------------------------------------------------------------------------
// coarse CG (relative residual tol, zero start).  Control block on the device:
// rr[2] (ping-pong by iteration parity), pAp, stop; ints: done, iter.
// Every kernel returns at once when done is set, so the host can queue
// iterations in batches and read the flag once per batch.
// ---------------------------------------------------------------------------
struct CCtl {
  double rr[2];
  double pAp;
  double stop;
  int done;
  int iter;
};

template <typename R>
__global__ void k_ccg_init(const typename CV<R>::T* rhs, typename CV<R>::T* x, typename CV<R>::T* r,
                           typename CV<R>::T* p, size_t nc, Reduction red) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v[1] = {0.0};
  if (t < nc) {
    const typename CV<R>::T b = rhs[t];
    x[t] = {0, 0};
    r[t] = b;
    p[t] = b;
    v[0] = (double)b.x * b.x + (double)b.y * b.y;
  }
  grid_reduce<1>(v, red);
}

__global__ void k_ccg_start(CCtl* ctl, double tol, int maxiter) {
  ctl->stop = tol * tol * ctl->rr[0];
  ctl->iter = 0;
  ctl->done = (ctl->rr[0] == 0.0 || maxiter <= 0) ? 1 : 0;
}

template <typename AT, typename R, int VJ>
__global__ void __launch_bounds__(256) k_ccg_apply(const AT* __restrict__ A, const int* __restrict__ cnbr, int n,
                                                   const typename CV<R>::T* __restrict__ p, typename CV<R>::T* wpart,
                                                   size_t nc, const CCtl* ctl, Reduction red) {
  if (ctl->done) return;
  double dv = 0.0;
  capply_body<AT, R, VJ>(A, cnbr, n, p, wpart, nc, &dv);
  double v[1] = {dv};
  grid_reduce<1>(v, red);
}

template <typename R>
__global__ void k_ccg_update(typename CV<R>::T* x, typename CV<R>::T* r, const typename CV<R>::T* p,
                             const typename CV<R>::T* w, size_t nc, const CCtl* ctl, int par, Reduction red) {
  if (ctl->done) return;
  const double alpha = ctl->pAp > 0 ? ctl->rr[par] / ctl->pAp : 0.0;
  const R al = (R)alpha;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v[1] = {0.0};
  if (t < nc) {
    typename CV<R>::T xv = x[t], rv = r[t];
    const typename CV<R>::T pv = p[t];
    typename CV<R>::T wv = w[t];
#pragma unroll
    for (int g = 1; g < CGROUPS; ++g) {
      wv.x += w[g * nc + t].x;
      wv.y += w[g * nc + t].y;
    }
    xv.x += al * pv.x;
    xv.y += al * pv.y;
    rv.x -= al * wv.x;
    rv.y -= al * wv.y;
    x[t] = xv;
    r[t] = rv;
    v[0] = (double)rv.x * rv.x + (double)rv.y * rv.y;
  }
  grid_reduce<1>(v, red);
}

template <typename R>
__global__ void k_ccg_p(typename CV<R>::T* p, const typename CV<R>::T* r, size_t nc, CCtl* ctl, int par,
                        int maxiter) {
  if (ctl->done) return;
  const double rr_old = ctl->rr[par], rr_new = ctl->rr[par ^ 1];
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) {
    const int it = ctl->iter + 1;
    ctl->iter = it;
    if (rr_new <= ctl->stop || it >= maxiter || !(rr_new == rr_new)) ctl->done = 1;
  }
  const R beta = (R)(rr_old > 0 ? rr_new / rr_old : 0.0);
  if (t < nc) {
    typename CV<R>::T pv = p[t];
    const typename CV<R>::T rv = r[t];
    pv.x = rv.x + beta * pv.x;
    pv.y = rv.y + beta * pv.y;
    p[t] = pv;
  }
}

template <typename AT, typename R>
static int coarse_cg_t(Ctx& c, Coarse& A, const void* rhs, void* sol, double tol, int maxiter) {
  using V = typename CV<R>::T;
  const size_t nc = A.Vc * A.nvec;
  A.work.ensure((2 + CGROUPS) * nc * sizeof(V));
  A.ctl.ensure(sizeof(CCtl));
  V* r = A.work.as<V>();
  V* p = r + nc;
  V* w = p + nc;   // CGROUPS partial products
  CCtl* ctl = A.ctl.as<CCtl>();
  const unsigned gv = (unsigned)((nc + 255) / 256);
  k_ccg_init<R><<<gv, 256, 0, c.stream>>>((const V*)rhs, (V*)sol, r, p, nc, make_reduction(c, gv, 1, &ctl->rr[0], 0));
  k_ccg_start<<<1, 1, 0, c.stream>>>(ctl, tol, maxiter);
  c.launches += 2;
  int queued = 0;
  int batch = std::max(1, A.last_iters);
  CCtl h{};
  while (true) {
    for (int b = 0; b < batch && queued < maxiter; ++b, ++queued) {
      const int par = queued & 1;
      const Reduction rd = make_reduction(c, (unsigned)(A.Vc * CGROUPS), 1, &ctl->pAp, 0);
      if (A.nvec % vec_width<AT>() == 0)
        k_ccg_apply<AT, R, vec_width<AT>()><<<(unsigned)(A.Vc * CGROUPS), 256, 0, c.stream>>>(
            A.A.as<AT>(), A.cnbr.as<int>(), A.nvec, p, w, nc, ctl, rd);
      else
        k_ccg_apply<AT, R, 1><<<(unsigned)(A.Vc * CGROUPS), 256, 0, c.stream>>>(A.A.as<AT>(), A.cnbr.as<int>(),
                                                                              A.nvec, p, w, nc, ctl, rd);
      k_ccg_update<R><<<gv, 256, 0, c.stream>>>((V*)sol, r, p, w, nc, ctl, par,
                                                make_reduction(c, gv, 1, &ctl->rr[par ^ 1], 0));
      k_ccg_p<R><<<gv, 256, 0, c.stream>>>(p, r, nc, ctl, par, maxiter);
      c.launches += 3;
    }
    HDCG_CUDA(cudaGetLastError());
    HDCG_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(CCtl), cudaMemcpyDeviceToHost, c.stream));
    HDCG_CUDA(cudaStreamSynchronize(c.stream));
    if (h.done || queued >= maxiter) break;
    batch = 2;
  }
  A.last_iters = std::max(1, h.iter);
  return h.iter;
}

// Single right-hand side with an FP16/FP32 operator: time eight iterations of the
// CUDA-core and of the tensor-core coarse CG once per operator, keep the faster.
static void tune_single(Ctx& c, Coarse& A, const void* rhs, void* sol) {
  coarse_tc_prepare(c, A);
  const int keep = A.last_iters;
  cudaEvent_t e[3];
  for (auto& ev : e) HDCG_CUDA(cudaEventCreate(&ev));
  A.last_iters = 8;
  auto core = [&] {
    if (A.prec == HDCG_F32) coarse_cg_t<float2, float>(c, A, rhs, sol, 1e-30, 8);
    else coarse_cg_t<__half2, float>(c, A, rhs, sol, 1e-30, 8);
  };
  core();
  coarse_cg_tc(c, A, 1, rhs, sol, 1e-30, 8);
  HDCG_CUDA(cudaEventRecord(e[0], c.stream));
  core();
  HDCG_CUDA(cudaEventRecord(e[1], c.stream));
  coarse_cg_tc(c, A, 1, rhs, sol, 1e-30, 8);
  HDCG_CUDA(cudaEventRecord(e[2], c.stream));
  HDCG_CUDA(cudaEventSynchronize(e[2]));
  float t_core = 0, t_tc = 0;
  HDCG_CUDA(cudaEventElapsedTime(&t_core, e[0], e[1]));
  HDCG_CUDA(cudaEventElapsedTime(&t_tc, e[1], e[2]));
  for (auto& ev : e) cudaEventDestroy(ev);
  A.tc_choice = t_tc < t_core ? 1 : 0;
  A.last_iters = keep;
}

bool coarse_use_tc_single(Ctx& c, Coarse& A) {
  if (!coarse_tc_supported(A)) return false;
  return A.tc_choice == 1;
}

int coarse_cg(Ctx& c, Coarse& A, const void* rhs, void* sol, double tol, int maxiter) {
  if (level2_active(A)) return level1_solve(c, A, 1, rhs, sol, tol, maxiter);
  if (A.defl.nd > 0) {
    if (coarse_tc_supported(A) && A.tc_choice < 0) tune_single(c, A, rhs, sol);
    return coarse_adef1(c, A, 1, rhs, sol, tol, maxiter);
  }
  if (coarse_tc_supported(A)) {
    if (A.tc_choice < 0) tune_single(c, A, rhs, sol);
    if (A.tc_choice == 1) return coarse_cg_tc(c, A, 1, rhs, sol, tol, maxiter);
  }
  if (A.prec == HDCG_F64) return coarse_cg_t<double2, double>(c, A, rhs, sol, tol, maxiter);
  if (A.prec == HDCG_F32) return coarse_cg_t<float2, float>(c, A, rhs, sol, tol, maxiter);
  return coarse_cg_t<__half2, float>(c, A, rhs, sol, tol, maxiter);
}

template <typename Ti, typename To>
__global__ void k_cvec_convert(const Ti* in, To* out, size_t n) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = {(decltype(out[t].x))in[t].x, (decltype(out[t].y))in[t].y};
}

void cvec_convert(Ctx& c, const void* in, int pin, void* out, int pout, size_t n) {
  const unsigned g = (unsigned)((n + 255) / 256);
  if (pin == pout) {
    HDCG_CUDA(cudaMemcpyAsync(out, in, n * (pin == HDCG_F64 ? 16 : 8), cudaMemcpyDeviceToDevice, c.stream));
    return;
  }
  if (pin == HDCG_F64) k_cvec_convert<double2, float2><<<g, 256, 0, c.stream>>>((const double2*)in, (float2*)out, n);
  else k_cvec_convert<float2, double2><<<g, 256, 0, c.stream>>>((const float2*)in, (double2*)out, n);
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}

template <typename AT>
__global__ void k_coarse_export(const AT* A, double2* out, int n, size_t Vc) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t per = (size_t)81 * n * n;
  if (t >= Vc * per) return;
  const size_t a = t / per;
  const int rem = (int)(t % per);
  const int l = rem / (n * n), j = (rem / n) % n, k = rem % n;
  const size_t src = ((a * 81 + l) * n + k) * n + j;  // internal [a][l][k][j]
  if constexpr (sizeof(AT) == 16) out[t] = ((const double2*)A)[src];
  else if constexpr (sizeof(AT) == 8) {
    const float2 v = ((const float2*)A)[src];
    out[t] = make_double2(v.x, v.y);
  } else {
    const float2 v = __half22float2(((const __half2*)A)[src]);
    out[t] = make_double2(v.x, v.y);
  }
}

// canonical [a][l][j][k] complex double -> internal [a][l][k][j] in the storage precision
template <typename AT>
__global__ void k_coarse_import(const double2* __restrict__ in, AT* A, int n, size_t Vc) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t per = (size_t)81 * n * n;
  if (t >= Vc * per) return;
  const size_t a = t / per;
  const int rem = (int)(t % per);
  const int l = rem / (n * n), j = (rem / n) % n, k = rem % n;
  const size_t dst = ((a * 81 + l) * n + k) * n + j;
  const double2 v = in[t];
  if constexpr (sizeof(AT) == 16) ((double2*)A)[dst] = v;
  else if constexpr (sizeof(AT) == 8) ((float2*)A)[dst] = make_float2((float)v.x, (float)v.y);
  else ((__half2*)A)[dst] = __halves2half2(__double2half(v.x), __double2half(v.y));
}

void coarse_import(Ctx& c, Coarse& A, const void* src, int on_device) {
  const size_t tot = A.Vc * 81 * A.nvec * A.nvec;
  DevMem d;
  const double2* in = static_cast<const double2*>(src);
  if (!on_device) {
    d.ensure(tot * sizeof(double2));
    HDCG_CUDA(cudaMemcpyAsync(d.p, src, tot * sizeof(double2), cudaMemcpyHostToDevice, c.stream));
    in = d.as<double2>();
  }
  const unsigned g = (unsigned)((tot + 255) / 256);
  if (A.prec == HDCG_F64) k_coarse_import<double2><<<g, 256, 0, c.stream>>>(in, A.A.as<double2>(), A.nvec, A.Vc);
  else if (A.prec == HDCG_F32) k_coarse_import<float2><<<g, 256, 0, c.stream>>>(in, A.A.as<float2>(), A.nvec, A.Vc);
  else {
    k_coarse_import<__half2><<<g, 256, 0, c.stream>>>(in, A.A.as<__half2>(), A.nvec, A.Vc);
    A.Aacc.ensure(tot * sizeof(float2));
    k_coarse_import<float2><<<g, 256, 0, c.stream>>>(in, A.Aacc.as<float2>(), A.nvec, A.Vc);
    ++c.launches;
  }
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
  A.tc_ready = false;
  A.tc_choice = -1;
  for (int& v : A.tc_cfg) v = 0;
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
}

void coarse_export(Ctx& c, const Coarse& A, void* host) {
  const size_t tot = A.Vc * 81 * A.nvec * A.nvec;
  DevMem d;
  d.ensure(tot * sizeof(double2));
  const unsigned g = (unsigned)((tot + 255) / 256);
  if (A.prec == HDCG_F64) k_coarse_export<double2><<<g, 256, 0, c.stream>>>(A.A.as<double2>(), d.as<double2>(), A.nvec, A.Vc);
  else if (A.prec == HDCG_F32) k_coarse_export<float2><<<g, 256, 0, c.stream>>>(A.A.as<float2>(), d.as<double2>(), A.nvec, A.Vc);
  else k_coarse_export<__half2><<<g, 256, 0, c.stream>>>(A.A.as<__half2>(), d.as<double2>(), A.nvec, A.Vc);
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
  HDCG_CUDA(cudaMemcpyAsync(host, d.p, tot * sizeof(double2), cudaMemcpyDeviceToHost, c.stream));
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
}

// ---------------------------------------------------------------------------
// Coarse stencil apply that allocates nothing (hdcg_coarse_apply_noalloc).
// Its scratch -- the coarse vectors in the working precision and the
// CGROUPS partial products -- lives in one file-scope device array of fixed
// size instead of memory obtained from cudaMalloc, for callers that must not
// allocate device memory on this path.  Every GPU that loads the library
// holds the array until the process exits.  All calls on a device share it
// and it keeps the previous call's contents; nothing in it needs to start at
// zero because every call overwrites all the bytes it reads.  Calls that
// overlap on the GPU (other streams, other host threads) race on it.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of the array on the current device.  The handle looks it up
// with that device current on its first no-alloc call (and again if the
// current device changes) and keeps it for its own lifetime: a handle never
// outlives the CUDA context it was created in, so the address cannot go stale
// the way a process-wide cache could after a device reset.
static char* noalloc_scratch(Ctx& c) {
  int dev = 0;
  HDCG_CUDA(cudaGetDevice(&dev));
  if (c.noalloc_addr == nullptr || c.noalloc_dev != dev) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      throw Error{HDCG_ERR_CUDA, std::string("cudaGetSymbolAddress of the no-alloc scratch: ") + cudaGetErrorString(e)};
    c.noalloc_addr = p;
    c.noalloc_dev = dev;
  }
  return reinterpret_cast<char*>(c.noalloc_addr);
}

size_t coarse_apply_noalloc_bytes(const Coarse& A) {
  const size_t nc = A.Vc * A.nvec;
  // FP64 vectors: the caller's buffers are used directly, scratch = partials;
  // FP32 vectors: converted x, y and the partials
  return A.vec_prec() == HDCG_F64 ? CGROUPS * nc * sizeof(double2) : (2 + CGROUPS) * nc * sizeof(float2);
}

template <typename AT, typename R>
static void coarse_apply_noalloc_t(Ctx& c, const Coarse& A, const void* x64, void* y64) {
  using V = typename CV<R>::T;
  const size_t nc = A.Vc * A.nvec;
  char* arena = noalloc_scratch(c);
  const unsigned gv = (unsigned)((nc + 255) / 256);
  const V* x;
  V* y;
  V* part;
  if (sizeof(V) == sizeof(double2)) {
    x = reinterpret_cast<const V*>(x64);
    y = reinterpret_cast<V*>(y64);
    part = reinterpret_cast<V*>(arena);
  } else {
    V* xs = reinterpret_cast<V*>(arena);
    V* ys = xs + nc;
    part = ys + nc;
    k_cvec_convert<double2, V><<<gv, 256, 0, c.stream>>>(reinterpret_cast<const double2*>(x64), xs, nc);
    ++c.launches;
    x = xs;
    y = ys;
  }
  if (A.nvec % vec_width<AT>() == 0)
    k_coarse_apply<AT, R, vec_width<AT>()><<<(unsigned)(A.Vc * CGROUPS), 256, 0, c.stream>>>(
        A.A.as<AT>(), A.cnbr.as<int>(), A.nvec, x, part, nc, 0, Reduction{});
  else
    k_coarse_apply<AT, R, 1><<<(unsigned)(A.Vc * CGROUPS), 256, 0, c.stream>>>(A.A.as<AT>(), A.cnbr.as<int>(),
                                                                              A.nvec, x, part, nc, 0, Reduction{});
  k_sum_groups<R><<<gv, 256, 0, c.stream>>>(part, y, nc);
  c.launches += 2;
  if (sizeof(V) != sizeof(double2)) {
    k_cvec_convert<V, double2><<<gv, 256, 0, c.stream>>>(y, reinterpret_cast<double2*>(y64), nc);
    ++c.launches;
  }
  HDCG_CUDA(cudaGetLastError());
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
}

void coarse_apply_noalloc(Ctx& c, const Coarse& A, const void* x64, void* y64) {
  HDCG_REQUIRE(A.nvec <= 64, HDCG_ERR_ARG, "nvec <= 64");
  const size_t need = coarse_apply_noalloc_bytes(A);
  if (need > NOALLOC_SCRATCH_BYTES)
    throw Error{HDCG_ERR_ARG, "coarse operator too large for the no-alloc scratch: needs " + std::to_string(need) +
                                  " bytes, limit " + std::to_string((size_t)NOALLOC_SCRATCH_BYTES) + " bytes"};
  if (A.prec == HDCG_F64) coarse_apply_noalloc_t<double2, double>(c, A, x64, y64);
  else if (A.prec == HDCG_F32) coarse_apply_noalloc_t<float2, float>(c, A, x64, y64);
  else coarse_apply_noalloc_t<__half2, float>(c, A, x64, y64);
}


// ---------------------------------------------------------------------------
// several right-hand sides (the batched solver).  Coarse vectors of R
// right-hand sides are stored [a][k][r] (right-hand side fastest).
// ---------------------------------------------------------------------------

// c[a][k][r] = <phi_k^a, v_r> for R fields v (one Gram pass reads phi once)
void restrict_multi(Ctx& c, const Subspace& s, const uint4* v, int vprec, int R, void* cvec, int cprec) {
  const size_t nc = s.Vc * s.nvec * (size_t)R;
  DevMem G;
  G.ensure(nc * sizeof(double2));
  block_gram(c, s, v, R, vprec, c.field_bytes(vprec) / 16, G.as<double2>(), (size_t)s.nvec * R, GramPhase{});
  cvec_convert(c, G.p, HDCG_F64, cvec, cprec, nc);
}

// out_r = f_r (add_r + sum_k c[b][k][r] phi_k)  (tile of all vectors in shared memory);
// the added field may be stored in a narrower precision Sa than the output
template <typename Sp, typename So, typename Rt, typename Sa>
__global__ void __launch_bounds__(256) k_prolong_multi(const uint4* phi, size_t pstride, int n, BlockArgs ba,
                                                       const typename CV<Rt>::T* __restrict__ cv, int R,
                                                       uint4* out, const uint4* add, size_t ostride, size_t astride,
                                                       const double* un_num, const double* un_den) {
  using Ro = typename Store<So>::real;
  using Ra = typename Store<Sa>::real;
  constexpr int C = Store<So>::chunks, P = Store<So>::per_chunk, PA = Store<Sa>::per_chunk;
  static_assert(PA >= P, "the added field's chunks hold at least one output chunk");
  extern __shared__ __align__(16) unsigned char smraw[];
  Rt* xs = reinterpret_cast<Rt*>(smraw);
  Rt* cs = xs + (size_t)n * TROW;    // [k][r] complex
  __shared__ Rt unscale[RMAX];
  const size_t b = blockIdx.x;
  for (int q = threadIdx.x; q < n * R; q += blockDim.x) {
    const typename CV<Rt>::T v = cv[b * n * R + q];
    cs[2 * q] = v.x;
    cs[2 * q + 1] = v.y;
  }
  if (threadIdx.x < RMAX)
    unscale[threadIdx.x] = (un_num && (int)threadIdx.x < R) ? (Rt)sqrt(un_den[threadIdx.x] / un_num[0]) : Rt(1);
  const int nsites = ba.spb * ba.Ls;
  const int units = R * TILE * C;
  for (int tile0 = 0; tile0 < nsites; tile0 += TILE) {
    __syncthreads();
    load_tile<Sp, Rt>(xs, phi, pstride, n, ba, b, tile0);
    __syncthreads();
    for (int u = threadIdx.x; u < units; u += blockDim.x) {
      const int t = u % TILE;
      const int ch = (u / TILE) % C;
      const int r = u / (C * TILE);
      Rt o[P];
#pragma unroll
      for (int i = 0; i < P; ++i) o[i] = 0;
      for (int k = 0; k < n; ++k) {
        const Rt cr = cs[2 * (k * R + r)], ci = cs[2 * (k * R + r) + 1];
        const Rt* xr = xs + k * TROW + t * 24 + ch * P;
#pragma unroll
        for (int i = 0; i < P; i += 2) {
          o[i] += cr * xr[i] - ci * xr[i + 1];
          o[i + 1] += cr * xr[i + 1] + ci * xr[i];
        }
      }
      const size_t site5 = block_site5(ba, b, tile0 + t);
      if (add) {
        // the P reals of this output chunk sit in chunk (ch P) / PA of the added field
        Ra av[PA];
        unpack(Sa{}, __ldg(add + r * astride + ((ch * P) / PA) * ba.n5 + site5), av);
        const int off = (ch * P) % PA;
#pragma unroll
        for (int i = 0; i < P; ++i) o[i] += (Rt)av[off + i];
      }
      const Rt f = unscale[r];
      Ro w[P];
#pragma unroll
      for (int i = 0; i < P; ++i) w[i] = (Ro)(f * o[i]);
      out[r * ostride + ch * ba.n5 + site5] = pack(So{}, w);
    }
  }
}

template <typename Sp, typename So, typename Rt, typename Sa>
static void launch_prolong_multi(Ctx& c, const Subspace& s, const void* cvec, int R, uint4* out, const uint4* add,
                                 size_t ostride, size_t astride, const double* un_num, const double* un_den) {
  const int n = s.nvec;
  const size_t sm = tile_smem<Rt>(n) + (size_t)n * R * 2 * sizeof(Rt);
  auto fn = k_prolong_multi<Sp, So, Rt, Sa>;
  set_smem_limit((const void*)fn, sm);
  fn<<<(unsigned)s.Vc, 256, sm, c.stream>>>(s.vecs.as<uint4>(), s.vec_bytes(c) / 16, n, block_args(c, s),
                                             (const typename CV<Rt>::T*)cvec, R, out, add, ostride, astride, un_num,
                                             un_den);
}

void prolong_multi(Ctx& c, const Subspace& s, const void* cvec, int cprec, int R, uint4* out, int oprec,
                   const uint4* add, int add_prec, const double* un_num, const double* un_den) {
  HDCG_REQUIRE((cprec == HDCG_F64) == (s.prec == HDCG_F64), HDCG_ERR_ARG,
               "coarse vectors are FP64 exactly when the subspace is FP64");
  HDCG_REQUIRE(R >= 1 && R <= RMAX, HDCG_ERR_ARG, "1..16 right-hand sides");
  if (add_prec < 0 || !add) add_prec = oprec;
  HDCG_REQUIRE(add_prec == oprec || (add_prec == HDCG_F16 && (oprec == HDCG_F32 || oprec == HDCG_F64)),
               HDCG_ERR_ARG, "prolongation: the added field is in the output precision or FP16");
  const size_t ostride = c.field_bytes(oprec) / 16, astride = c.field_bytes(add_prec) / 16;
  DISPATCH_SUB(s.prec, Sp, {
    using Rt = typename std::conditional<std::is_same<Sp, f64_t>::value, double, float>::type;
    if (add_prec != oprec) {
      if (oprec == HDCG_F32)
        launch_prolong_multi<Sp, f32_t, Rt, f16_t>(c, s, cvec, R, out, add, ostride, astride, un_num, un_den);
      else
        launch_prolong_multi<Sp, f64_t, Rt, f16_t>(c, s, cvec, R, out, add, ostride, astride, un_num, un_den);
    } else {
      DISPATCH_PREC(oprec, So, {
        launch_prolong_multi<Sp, So, Rt, So>(c, s, cvec, R, out, add, ostride, astride, un_num, un_den);
      });
    }
  });
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}

// Y[a][j][r] = sum_l sum_k A[a][l][k][j] X[a+l][k][r] for R right-hand sides.
// Same warp layout as capply_body; every lane keeps VJ x R accumulators and
// reads A once for all right-hand sides.  Per-rhs partial dots Re<X_r, Y_r>
// of this CGROUPS slice go to dot_out[r].
template <typename AT, typename R_, int VJ>
__device__ __forceinline__ void capply_multi_body(const AT* __restrict__ A, const int* __restrict__ cnbr, int n,
                                                  int R, const typename CV<R_>::T* __restrict__ x,
                                                  typename CV<R_>::T* ypart, size_t nc, double* dot_out,
                                                  typename CV<R_>::T* sred, R_ shift) {
  using V = typename CV<R_>::T;
  const size_t a = blockIdx.x / CGROUPS;
  const int g = blockIdx.x % CGROUPS;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int NJ = n / VJ;
  const int KS = NJ <= 32 ? 32 / NJ : 1;
  const int ks = NJ <= 32 ? lane / NJ : 0;
  const int jp0 = NJ <= 32 ? lane % NJ : lane;
  const bool on0 = ks < KS && jp0 < NJ;
  const bool on1 = NJ > 32 && lane + 32 < NJ;
  const int l0 = g * 27, l1 = l0 + 27;
  R_ sr[2 * VJ][RMAX], si[2 * VJ][RMAX];
#pragma unroll
  for (int q = 0; q < 2 * VJ; ++q)
#pragma unroll
    for (int r = 0; r < RMAX; ++r) sr[q][r] = si[q][r] = 0;
  for (int l = l0 + w; l < l1; l += CWARPS) {
    const int nb = __ldg(cnbr + a * 81 + l);
    const AT* blk = A + ((a * 81 + l) * n) * n;
    const V* xv = x + (size_t)nb * n * R;
    for (int k = ks; k < n; k += KS) {
      R_ ar[2 * VJ], ai[2 * VJ];
#pragma unroll
      for (int q = 0; q < 2 * VJ; ++q) ar[q] = ai[q] = 0;
      if (on0) ld_a_vec<AT, R_, VJ>(blk + (size_t)k * n + jp0 * VJ, ar, ai);
      if (on1) ld_a_vec<AT, R_, VJ>(blk + (size_t)k * n + (jp0 + 32) * VJ, ar + VJ, ai + VJ);
#pragma unroll
      for (int r = 0; r < RMAX; ++r) {
        if (r < R) {
          const V xk = xv[(size_t)k * R + r];
#pragma unroll
          for (int q = 0; q < 2 * VJ; ++q) {
            sr[q][r] += ar[q] * xk.x - ai[q] * xk.y;
            si[q][r] += ar[q] * xk.y + ai[q] * xk.x;
          }
        }
      }
    }
  }
  if (NJ <= 32) {
    for (int d = 1; d < KS; d <<= 1) {
#pragma unroll
      for (int q = 0; q < VJ; ++q)
#pragma unroll
        for (int r = 0; r < RMAX; ++r) {
          const R_ tr = __shfl_down_sync(FULL_MASK, sr[q][r], d * NJ);
          const R_ ti = __shfl_down_sync(FULL_MASK, si[q][r], d * NJ);
          if ((ks & (2 * d - 1)) == 0 && ks + d < KS) {
            sr[q][r] += tr;
            si[q][r] += ti;
          }
        }
    }
  }
  // sred: [CWARPS][n][R] in the working precision
  if (ks == 0 && jp0 < NJ)
#pragma unroll
    for (int q = 0; q < VJ; ++q)
      for (int r = 0; r < R; ++r)
        sred[((size_t)w * n + jp0 * VJ + q) * R + r] = {sr[q][r], si[q][r]};
  if (on1)
#pragma unroll
    for (int q = 0; q < VJ; ++q)
      for (int r = 0; r < R; ++r)
        sred[((size_t)w * n + (jp0 + 32) * VJ + q) * R + r] = {sr[VJ + q][r], si[VJ + q][r]};
  __syncthreads();
  for (int r = 0; r < RMAX; ++r) dot_out[r] = 0.0;
  for (int o = threadIdx.x; o < n * R; o += blockDim.x) {
    R_ tr = 0, ti = 0;
#pragma unroll
    for (int q = 0; q < CWARPS; ++q) {
      const V v = sred[(size_t)q * n * R + o];
      tr += v.x;
      ti += v.y;
    }
    const V xa = x[a * n * R + o];
    if (g == 0) {   // (A + shift) x: the shift enters once, with the first group
      tr += shift * xa.x;
      ti += shift * xa.y;
    }
    ypart[g * nc + a * n * R + o] = {tr, ti};
    const int r = o % R;
#pragma unroll
    for (int rr = 0; rr < RMAX; ++rr)
      if (rr == r) dot_out[rr] += (double)xa.x * tr + (double)xa.y * ti;
  }
}

struct CCtlM {
  double rr[2][RMAX];
  double pAp[RMAX];
  double stop[RMAX];
  int done[RMAX];
  int iter;
  int all_done;
};

template <typename AT, typename R_, int VJ>
__global__ void __launch_bounds__(256) k_capply_multi(const AT* __restrict__ A, const int* __restrict__ cnbr, int n,
                                                      int R, const typename CV<R_>::T* __restrict__ x,
                                                      typename CV<R_>::T* ypart, size_t nc, const int* skip,
                                                      Reduction red, R_ shift) {
  extern __shared__ __align__(16) unsigned char smraw[];
  if (skip && *skip) return;
  double dot[RMAX];
  capply_multi_body<AT, R_, VJ>(A, cnbr, n, R, x, ypart, nc, dot, reinterpret_cast<typename CV<R_>::T*>(smraw),
                                shift);
  if (red.result) grid_reduce<RMAX>(dot, red, R);
}

template <typename R_>
__global__ void k_ccgm_init(const typename CV<R_>::T* rhs, typename CV<R_>::T* x, typename CV<R_>::T* r,
                            typename CV<R_>::T* p, size_t ne, int R, Reduction red) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // coarse site-vector (a, k)
  double v[RMAX];
#pragma unroll
  for (int q = 0; q < RMAX; ++q) v[q] = 0.0;
  if (t < ne) {
#pragma unroll
    for (int q = 0; q < RMAX; ++q) {
      if (q < R) {
        const typename CV<R_>::T b = rhs[t * R + q];
        x[t * R + q] = {0, 0};
        r[t * R + q] = b;
        p[t * R + q] = b;
        v[q] = (double)b.x * b.x + (double)b.y * b.y;
      }
    }
  }
  grid_reduce<RMAX>(v, red, R);
}

__global__ void k_ccgm_start(CCtlM* ctl, int R, double tol, int maxiter) {
  int all = 1;
  for (int q = 0; q < R; ++q) {
    ctl->stop[q] = tol * tol * ctl->rr[0][q];
    ctl->done[q] = (ctl->rr[0][q] == 0.0 || maxiter <= 0) ? 1 : 0;
    all &= ctl->done[q];
  }
  ctl->iter = 0;
  ctl->all_done = all;
}

template <typename R_>
__global__ void k_ccgm_update(typename CV<R_>::T* x, typename CV<R_>::T* r, const typename CV<R_>::T* p,
                              const typename CV<R_>::T* w, size_t ne, int R, size_t nc, const CCtlM* ctl, int par,
                              Reduction red) {
  if (ctl->all_done) return;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v[RMAX];
#pragma unroll
  for (int q = 0; q < RMAX; ++q) v[q] = 0.0;
  if (t < ne) {
#pragma unroll
    for (int q = 0; q < RMAX; ++q) {
      if (q < R) {
        const double pap = ctl->pAp[q];
        const R_ al = (R_)((!ctl->done[q] && pap > 0) ? ctl->rr[par][q] / pap : 0.0);
        const size_t e = t * R + q;
        typename CV<R_>::T xv = x[e], rv = r[e];
        const typename CV<R_>::T pv = p[e];
        typename CV<R_>::T wv = w[e];
#pragma unroll
        for (int g = 1; g < CGROUPS; ++g) {
          wv.x += w[g * nc + e].x;
          wv.y += w[g * nc + e].y;
        }
        xv.x += al * pv.x;
        xv.y += al * pv.y;
        rv.x -= al * wv.x;
        rv.y -= al * wv.y;
        x[e] = xv;
        r[e] = rv;
        v[q] = (double)rv.x * rv.x + (double)rv.y * rv.y;
      }
    }
  }
  grid_reduce<RMAX>(v, red, R);
}

template <typename R_>
__global__ void k_ccgm_p(typename CV<R_>::T* p, const typename CV<R_>::T* r, size_t ne, int R, CCtlM* ctl, int par,
                         int maxiter) {
  if (ctl->all_done) return;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < ne) {
#pragma unroll
    for (int q = 0; q < RMAX; ++q) {
      if (q < R && !ctl->done[q]) {
        const double ro = ctl->rr[par][q], rn = ctl->rr[par ^ 1][q];
        const R_ beta = (R_)(ro > 0 ? rn / ro : 0.0);
        const size_t e = t * R + q;
        typename CV<R_>::T pv = p[e];
        const typename CV<R_>::T rv = r[e];
        pv.x = rv.x + beta * pv.x;
        pv.y = rv.y + beta * pv.y;
        p[e] = pv;
      }
    }
  }
}

// convergence bookkeeping after an iteration (one thread; ordered after k_ccgm_p)
__global__ void k_ccgm_check(CCtlM* ctl, int R, int par, int maxiter) {
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

template <typename AT, typename R_>
static int coarse_cg_multi_t(Ctx& c, Coarse& A, int R, const void* rhs, void* sol, double tol, int maxiter,
                             double shift) {
  using V = typename CV<R_>::T;
  const size_t ne = A.Vc * A.nvec;   // coarse site-vector elements per right-hand side
  const size_t nc = ne * R;
  A.work.ensure((2 + CGROUPS) * nc * sizeof(V));
  A.ctl.ensure(sizeof(CCtlM));
  V* r = A.work.as<V>();
  V* p = r + nc;
  V* w = p + nc;
  CCtlM* ctl = A.ctl.as<CCtlM>();
  const unsigned ge = (unsigned)((ne + 255) / 256);
  const unsigned ga = (unsigned)(A.Vc * CGROUPS);
  const size_t sm = (size_t)CWARPS * A.nvec * R * sizeof(V);
  const bool vec = A.nvec % vec_width<AT>() == 0;
  auto fn = vec ? k_capply_multi<AT, R_, vec_width<AT>()> : k_capply_multi<AT, R_, 1>;
  set_smem_limit((const void*)fn, sm);
  k_ccgm_init<R_><<<ge, 256, 0, c.stream>>>((const V*)rhs, (V*)sol, r, p, ne, R,
                                            make_reduction(c, ge, RMAX, &ctl->rr[0][0], 0));
  k_ccgm_start<<<1, 1, 0, c.stream>>>(ctl, R, tol, maxiter);
  c.launches += 2;
  int queued = 0;
  int batch = std::max(1, A.last_iters);
  CCtlM h{};
  while (true) {
    for (int bq = 0; bq < batch && queued < maxiter; ++bq, ++queued) {
      const int par = queued & 1;
      fn<<<ga, 256, sm, c.stream>>>(A.A.as<AT>(), A.cnbr.as<int>(), A.nvec, R, p, w, nc, &ctl->all_done,
                                    make_reduction(c, ga, RMAX, &ctl->pAp[0], 0), (R_)shift);
      k_ccgm_update<R_><<<ge, 256, 0, c.stream>>>((V*)sol, r, p, w, ne, R, nc, ctl, par,
                                                  make_reduction(c, ge, RMAX, &ctl->rr[par ^ 1][0], 0));
      k_ccgm_p<R_><<<ge, 256, 0, c.stream>>>(p, r, ne, R, ctl, par, maxiter);
      k_ccgm_check<<<1, 1, 0, c.stream>>>(ctl, R, par, maxiter);
      c.launches += 4;
    }
    HDCG_CUDA(cudaGetLastError());
    HDCG_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(CCtlM), cudaMemcpyDeviceToHost, c.stream));
    HDCG_CUDA(cudaStreamSynchronize(c.stream));
    if (h.all_done || queued >= maxiter) break;
    batch = 2;
  }
  A.last_iters = std::max(1, h.iter);
  return h.iter;
}

int coarse_cg_multi(Ctx& c, Coarse& A, int R, const void* rhs, void* sol, double tol, int maxiter, double shift,
                    bool deflate) {
  HDCG_REQUIRE(R >= 1 && R <= RMAX, HDCG_ERR_ARG, "1..16 right-hand sides");
  if (deflate && shift == 0.0 && level2_active(A)) return level1_solve(c, A, R, rhs, sol, tol, maxiter);
  if (deflate && A.defl.nd > 0 && shift == 0.0) return coarse_adef1(c, A, R, rhs, sol, tol, maxiter);
  if (coarse_tc_supported(A)) return coarse_cg_tc(c, A, R, rhs, sol, tol, maxiter, shift);
  if (A.prec == HDCG_F64) return coarse_cg_multi_t<double2, double>(c, A, R, rhs, sol, tol, maxiter, shift);
  if (A.prec == HDCG_F32) return coarse_cg_multi_t<float2, float>(c, A, R, rhs, sol, tol, maxiter, shift);
  return coarse_cg_multi_t<__half2, float>(c, A, R, rhs, sol, tol, maxiter, shift);
}

// single right-hand side, skipped while *skip is nonzero
template <typename AT, typename R, int VJ>
__global__ void __launch_bounds__(256) k_capply_skip(const AT* __restrict__ A, const int* __restrict__ cnbr, int n,
                                                     const typename CV<R>::T* __restrict__ x,
                                                     typename CV<R>::T* ypart, size_t nc, const int* skip,
                                                     Reduction red) {
  if (skip && *skip) return;
  double dv = 0.0;
  capply_body<AT, R, VJ>(A, cnbr, n, x, ypart, nc, &dv);
  double v[1] = {dv};
  grid_reduce<1>(v, red);
}

template <typename AT>
static int coarse_apply_partials_t(Ctx& c, const Coarse& A, int R, const float2* p, float2* wpart, const int* skip,
                                   double* pAp) {
  const size_t nc = A.Vc * A.nvec * (size_t)R;
  const unsigned ga = (unsigned)(A.Vc * CGROUPS);
  const bool vec = A.nvec % vec_width<AT>() == 0;
  if (R == 1) {
    auto fn = vec ? k_capply_skip<AT, float, vec_width<AT>()> : k_capply_skip<AT, float, 1>;
    fn<<<ga, 256, 0, c.stream>>>(A.A.as<AT>(), A.cnbr.as<int>(), A.nvec, p, wpart, nc, skip,
                                 make_reduction(c, ga, 1, pAp, 0));
  } else {
    const size_t sm = (size_t)CWARPS * A.nvec * R * sizeof(float2);
    auto fn = vec ? k_capply_multi<AT, float, vec_width<AT>()> : k_capply_multi<AT, float, 1>;
    set_smem_limit((const void*)fn, sm);
    fn<<<ga, 256, sm, c.stream>>>(A.A.as<AT>(), A.cnbr.as<int>(), A.nvec, R, p, wpart, nc, skip,
                                  make_reduction(c, ga, RMAX, pAp, 0), 0.f);
  }
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
  return CGROUPS;
}

int coarse_apply_partials(Ctx& c, const Coarse& A, int R, const float2* p, float2* wpart, const int* skip,
                          double* pAp) {
  HDCG_REQUIRE(A.prec == HDCG_F32 || A.prec == HDCG_F16, HDCG_ERR_ARG, "FP32 or FP16 coarse operator");
  if (A.prec == HDCG_F32) return coarse_apply_partials_t<float2>(c, A, R, p, wpart, skip, pAp);
  return coarse_apply_partials_t<__half2>(c, A, R, p, wpart, skip, pAp);
}

// Y = A X for R right-hand sides (canonical [a][k][r] complex double in and out)
template <typename AT, typename R_>
static void coarse_apply_multi_t(Ctx& c, const Coarse& A, int R, const void* x, void* y) {
  using V = typename CV<R_>::T;
  const size_t nc = A.Vc * A.nvec * (size_t)R;
  DevMem tmp;
  tmp.ensure((2 + CGROUPS) * nc * sizeof(V));
  V* xi = tmp.as<V>();
  V* yi = xi + nc;
  V* part = yi + nc;
  const int vp = A.vec_prec();
  cvec_convert(c, x, HDCG_F64, xi, vp, nc);
  const size_t sm = (size_t)CWARPS * A.nvec * R * sizeof(V);
  const bool vec = A.nvec % vec_width<AT>() == 0;
  auto fn = vec ? k_capply_multi<AT, R_, vec_width<AT>()> : k_capply_multi<AT, R_, 1>;
  set_smem_limit((const void*)fn, sm);
  Reduction none{};
  fn<<<(unsigned)(A.Vc * CGROUPS), 256, sm, c.stream>>>(A.A.as<AT>(), A.cnbr.as<int>(), A.nvec, R, xi, part, nc,
                                                         nullptr, none, (R_)0);
  k_sum_groups<R_><<<(unsigned)((nc + 255) / 256), 256, 0, c.stream>>>(part, yi, nc);
  c.launches += 2;
  cvec_convert(c, yi, vp, y, HDCG_F64, nc);
  HDCG_CUDA(cudaGetLastError());
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
}

void coarse_apply_multi(Ctx& c, const Coarse& A, int R, const void* x, void* y) {
  HDCG_REQUIRE(R >= 1 && R <= RMAX, HDCG_ERR_ARG, "1..16 right-hand sides");
  if (A.prec == HDCG_F64) coarse_apply_multi_t<double2, double>(c, A, R, x, y);
  else if (A.prec == HDCG_F32) coarse_apply_multi_t<float2, float>(c, A, R, x, y);
  else coarse_apply_multi_t<__half2, float>(c, A, R, x, y);
}

}  // namespace hdcg
