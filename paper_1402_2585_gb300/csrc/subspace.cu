// Subspace generation by a rational low-pass filter (Sec. 4.2, Eq. ratfilt,
// Table FineSubspaceParams).
//
// Every subspace vector starts from 4D Gaussian noise xi placed on the
// physical components of the walls, P_- xi at s = 0 and P_+ xi at s = Ls - 1
// (the components the mass term of P_s couples), and is filtered by
//   phi = prod_{i < order} (H + lam + i eps)^-1 eta = sum_i c_i (H + sigma_i)^-1 eta,
// c_i = prod_{j != i} 1 / (sigma_j - sigma_i) (partial fractions), with all
// order systems solved from one Krylov space by multi-shift CG: CG on the
// smallest shift sigma_0 = lam, whose residual polynomial R_k gives every
// shifted residual as r_k / R_k(-delta_i), delta_i = sigma_i - sigma_0, through
// the three-term recurrence R_{k+1}(t) = (1 - alpha_k t + g_k) R_k(t) -
// g_k R_{k-1}(t), g_k = alpha_k beta_{k-1} / alpha_{k-1}.  SubspaceSurfaceDepth
// keeps only the s-slices within depth of a wall.  Block Gram-Schmidt follows.
// The scalars of the recurrences live on the host (two reads per iteration,
// set-up only); fields are FP64 for an FP64 subspace, FP32 otherwise.
#include <cmath>
#include <vector>

#include "coarse.cuh"

namespace hdcg {

namespace {

constexpr int MSH_MAX = 8;   // shifts

__device__ __forceinline__ uint64_t smix(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// complex Gaussian number e (E|z|^2 = 1) of the splitmix64 stream seed, Box-Muller
__device__ __forceinline__ double2 cnormal(uint64_t seed, uint64_t e) {
  const double u1 = ((double)(smix(seed, 2 * e) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  const double u2 = ((double)(smix(seed, 2 * e + 1) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  const double r = sqrt(-2.0 * log(u1)) * 0.70710678118654752440;
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  return make_double2(r * cs, r * sn);
}

// field k: xi(k, x) (canonical order [k][x][spin][colour]) as P_- xi at s = 0
// and P_+ xi at s = Ls - 1, zero elsewhere (chiral basis: P_+ keeps spins 0, 1)
template <typename S>
__global__ void k_wall_noise(uint4* f, size_t n5, int lslog2, int Ls, int k, uint64_t seed) {
  using R = typename Store<S>::real;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n5) return;
  const size_t x = t >> lslog2;
  const int s = (int)(t & (Ls - 1));
  const size_t n4 = n5 >> lslog2;
  R v[24];
#pragma unroll
  for (int i = 0; i < 24; ++i) v[i] = 0;
  if (s == 0 || s == Ls - 1) {
    const int sp0 = s == 0 ? 2 : 0;
    for (int sp = sp0; sp < sp0 + 2; ++sp)
      for (int col = 0; col < 3; ++col) {
        const double2 z = cnormal(seed, (((size_t)k * n4 + x) * 4 + sp) * 3 + col);
        v[(sp * 3 + col) * 2] = (R)z.x;
        v[(sp * 3 + col) * 2 + 1] = (R)z.y;
      }
  }
  store_spinor<S, R>(f, t, n5, v);
}

struct ShiftCoef {
  double a[MSH_MAX];
};

// x_i += a_i p_i (i < ns); r -= alpha w; |r|^2
template <typename S>
__global__ void k_msh_x(uint4* xs, uint4* ps, size_t fs, int ns, ShiftCoef ca, uint4* r, const uint4* __restrict__ w,
                        double alpha, size_t n5, Reduction red) {
  using R = typename Store<S>::real;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v[1] = {0.0};
  if (t < n5) {
    R a[24], b[24];
    for (int i = 0; i < ns; ++i) {
      load_spinor<S, R>(xs + i * fs, t, n5, a);
      load_spinor<S, R>(ps + i * fs, t, n5, b);
      const R c = (R)ca.a[i];
#pragma unroll
      for (int e = 0; e < 24; ++e) a[e] += c * b[e];
      store_spinor<S, R>(xs + i * fs, t, n5, a);
    }
    load_spinor<S, R>(r, t, n5, a);
    load_spinor<S, R>(w, t, n5, b);
    const R al = (R)alpha;
    R s2 = 0;
#pragma unroll
    for (int e = 0; e < 24; ++e) {
      a[e] -= al * b[e];
      s2 += a[e] * a[e];
    }
    store_spinor<S, R>(r, t, n5, a);
    v[0] = (double)s2;
  }
  grid_reduce<1>(v, red);
}

// p_i = c_i r + d_i p_i (i < ns); pb = r + beta pb
template <typename S>
__global__ void k_msh_p(uint4* ps, size_t fs, int ns, ShiftCoef cc, ShiftCoef cd, const uint4* __restrict__ r,
                        uint4* pb, double beta, size_t n5) {
  using R = typename Store<S>::real;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n5) return;
  R rv[24], b[24];
  load_spinor<S, R>(r, t, n5, rv);
  for (int i = 0; i < ns; ++i) {
    load_spinor<S, R>(ps + i * fs, t, n5, b);
    const R c = (R)cc.a[i], d = (R)cd.a[i];
#pragma unroll
    for (int e = 0; e < 24; ++e) b[e] = c * rv[e] + d * b[e];
    store_spinor<S, R>(ps + i * fs, t, n5, b);
  }
  load_spinor<S, R>(pb, t, n5, b);
  const R be = (R)beta;
#pragma unroll
  for (int e = 0; e < 24; ++e) b[e] = rv[e] + be * b[e];
  store_spinor<S, R>(pb, t, n5, b);
}

// out (precision So) = sum_i c_i x_i, the s-slices deeper than depth from both walls zeroed
template <typename S, typename So>
__global__ void k_msh_combine(const uint4* __restrict__ xs, size_t fs, int ns, ShiftCoef cc, uint4* out, size_t n5,
                              int Ls, int depth) {
  using R = typename Store<S>::real;
  using Ro = typename Store<So>::real;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n5) return;
  const int s = (int)(t % Ls);
  const bool keep = depth <= 0 || s < depth || s >= Ls - depth;
  double acc[24];
#pragma unroll
  for (int e = 0; e < 24; ++e) acc[e] = 0.0;
  if (keep) {
    R b[24];
    for (int i = 0; i < ns; ++i) {
      load_spinor<S, R>(xs + i * fs, t, n5, b);
#pragma unroll
      for (int e = 0; e < 24; ++e) acc[e] += cc.a[i] * (double)b[e];
    }
  }
  Ro o[24];
#pragma unroll
  for (int e = 0; e < 24; ++e) o[e] = (Ro)acc[e];
  store_spinor<So, Ro>(out, t, n5, o);
}

template <typename S>
__global__ void k_msh_dot(const uint4* __restrict__ a, const uint4* __restrict__ b, size_t n5, Reduction red) {
  using R = typename Store<S>::real;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v[1] = {0.0};
  if (t < n5) {
    R x[24], y[24];
    load_spinor<S, R>(a, t, n5, x);
    load_spinor<S, R>(b, t, n5, y);
    R s = 0;
#pragma unroll
    for (int e = 0; e < 24; ++e) s += x[e] * y[e];
    v[0] = (double)s;
  }
  grid_reduce<1>(v, red);
}

// out (precision So) = the field of a handle with fifth extent Ls1 <= Ls placed
// into Ls: slices s < ceil(Ls1 / 2) stay at s, the others move to s + Ls - Ls1
// (each keeps its distance to its wall), the bulk between is zero
template <typename Si, typename So>
__global__ void k_promote(const uint4* __restrict__ in, size_t n51, int Ls1, uint4* out, size_t n5, int Ls,
                          int lslog2, size_t nf) {
  using Ri = typename Store<Si>::real;
  using Ro = typename Store<So>::real;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n5 * nf) return;
  const size_t f = t / n5, site5 = t % n5;
  const size_t x = site5 >> lslog2;
  const int s = (int)(site5 & (Ls - 1));
  const int h = (Ls1 + 1) / 2;
  int s1 = -1;
  if (s < h) s1 = s;
  else if (s >= Ls - (Ls1 - h)) s1 = s - (Ls - Ls1);
  Ro o[24];
#pragma unroll
  for (int e = 0; e < 24; ++e) o[e] = 0;
  if (s1 >= 0) {
    Ri v[24];
    load_spinor<Si, Ri>(in + f * n51 * Store<Si>::chunks, x * Ls1 + s1, n51, v);
#pragma unroll
    for (int e = 0; e < 24; ++e) o[e] = (Ro)v[e];
  }
  store_spinor<So, Ro>(out + f * n5 * Store<So>::chunks, site5, n5, o);
}

template <typename S>
__global__ void k_surface_truncate(uint4* f, size_t n5, int Ls, size_t nf, int depth) {
  using R = typename Store<S>::real;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n5 * nf) return;
  const size_t site5 = t % n5;
  const int s = (int)(site5 % Ls);
  if (s < depth || s >= Ls - depth) return;
  R z[24];
#pragma unroll
  for (int e = 0; e < 24; ++e) z[e] = 0;
  store_spinor<S, R>(f + (t / n5) * n5 * Store<S>::chunks, site5, n5, z);
}

}  // namespace

void rational_filter_shifts(double lam, double eps, int order, std::vector<double>& sig, std::vector<double>& c) {
  sig.resize(order);
  c.resize(order);
  for (int i = 0; i < order; ++i) sig[i] = lam + i * eps;
  for (int i = 0; i < order; ++i) {
    double w = 1.0;
    for (int j = 0; j < order; ++j)
      if (j != i) w /= (sig[j] - sig[i]);
    c[i] = w;
  }
}

template <typename S>
static int msh_filter(Ctx& c, int wp, const uint4* eta, uint4* xs, uint4* ps, uint4* r, uint4* pb, uint4* w,
                      const std::vector<double>& sig, double tol, int maxiter, double* dscal) {
  const int ns = (int)sig.size();
  const size_t fs = c.field_bytes(wp) / 16;
  const unsigned g = (unsigned)((c.n5 + 255) / 256);
  const double s0 = sig[0];
  std::vector<double> delta(ns);
  for (int i = 0; i < ns; ++i) delta[i] = sig[i] - s0;
  HDCG_CUDA(cudaMemsetAsync(xs, 0, c.field_bytes(wp) * ns, c.stream));
  for (int i = 0; i < ns; ++i)
    HDCG_CUDA(cudaMemcpyAsync(ps + i * fs, eta, c.field_bytes(wp), cudaMemcpyDeviceToDevice, c.stream));
  HDCG_CUDA(cudaMemcpyAsync(r, eta, c.field_bytes(wp), cudaMemcpyDeviceToDevice, c.stream));
  HDCG_CUDA(cudaMemcpyAsync(pb, eta, c.field_bytes(wp), cudaMemcpyDeviceToDevice, c.stream));
  k_msh_dot<S><<<g, 256, 0, c.stream>>>(eta, eta, c.n5, make_reduction(c, g, 1, dscal, 0));
  ++c.launches;
  double rr = 0;
  HDCG_CUDA(cudaMemcpyAsync(&rr, dscal, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
  const double bb = rr;
  if (bb == 0.0) return 0;
  std::vector<double> Rp(ns, 1.0), Rc(ns, 1.0), Rn(ns);
  double alpha_prev = 1.0, beta_prev = 0.0;
  int it = 0;
  while (it < maxiter) {
    apply_mdagm(c, wp, pb, w, nullptr, 1.0, s0, pb);   // w = (H + sigma_0) pb
    k_msh_dot<S><<<g, 256, 0, c.stream>>>(pb, w, c.n5, make_reduction(c, g, 1, dscal, 0));
    ++c.launches;
    double pw = 0;
    HDCG_CUDA(cudaMemcpyAsync(&pw, dscal, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    HDCG_CUDA(cudaStreamSynchronize(c.stream));
    HDCG_REQUIRE(std::isfinite(pw) && pw > 0, HDCG_ERR_BREAKDOWN, "multi-shift CG: (p, (H + sigma) p) <= 0");
    const double alpha = rr / pw;
    const double gk = alpha * beta_prev / alpha_prev;
    ShiftCoef ca{};
    for (int i = 0; i < ns; ++i) {
      Rn[i] = (1.0 + alpha * delta[i] + gk) * Rc[i] - gk * Rp[i];
      ca.a[i] = alpha * Rc[i] / Rn[i];
    }
    k_msh_x<S><<<g, 256, 0, c.stream>>>(xs, ps, fs, ns, ca, r, w, alpha, c.n5, make_reduction(c, g, 1, dscal, 0));
    ++c.launches;
    double rr_new = 0;
    HDCG_CUDA(cudaMemcpyAsync(&rr_new, dscal, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    HDCG_CUDA(cudaStreamSynchronize(c.stream));
    HDCG_REQUIRE(std::isfinite(rr_new), HDCG_ERR_NONFINITE, "multi-shift CG: non-finite residual");
    const double beta = rr_new / rr;
    ++it;
    ShiftCoef cc{}, cd{};
    for (int i = 0; i < ns; ++i) {
      const double ratio = Rc[i] / Rn[i];
      cc.a[i] = 1.0 / Rn[i];
      cd.a[i] = beta * ratio * ratio;
    }
    k_msh_p<S><<<g, 256, 0, c.stream>>>(ps, fs, ns, cc, cd, r, pb, beta, c.n5);
    HDCG_CUDA(cudaGetLastError());
    ++c.launches;
    Rp = Rc;
    Rc = Rn;
    alpha_prev = alpha;
    beta_prev = beta;
    rr = rr_new;
    if (rr <= tol * tol * bb) break;
  }
  return it;
}

// a 16-bit subspace is built in FP32 and rounded once at the end (the block
// pieces of a filtered subspace are nearly dependent before the block
// orthonormalisation separates them; 16-bit storage would blur them)
static void round_to_f16(Ctx& c, Subspace& s) {
  DevMem v32;
  std::swap(v32.p, s.vecs.p);
  std::swap(v32.bytes, s.vecs.bytes);
  s.prec = HDCG_F16;
  s.vecs.ensure((size_t)s.nvec * s.vec_bytes(c));
  convert_field(c, v32.as<uint4>(), HDCG_F32, s.vecs.as<uint4>(), HDCG_F16, s.nvec);
  block_orthonormalise(c, s);
}

static void truncate_surface(Ctx& c, Subspace& s, int depth) {
  if (depth <= 0 || 2 * depth >= c.Ls) return;
  const size_t n = c.n5 * s.nvec;
  DISPATCH_SUB(s.prec, S, {
    k_surface_truncate<S><<<(unsigned)((n + 255) / 256), 256, 0, c.stream>>>(s.vecs.as<uint4>(), c.n5, c.Ls, s.nvec,
                                                                              depth);
  });
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
}

static void check_filter(const hdcg_subspace_params& p) {
  HDCG_REQUIRE(p.filter_order >= 1 && p.filter_order <= MSH_MAX, HDCG_ERR_ARG, "filter order must be 1..8");
  HDCG_REQUIRE(p.filter_order == 1 || p.filter_eps > 0.0, HDCG_ERR_ARG, "the filter's shifts must differ (eps > 0)");
  HDCG_REQUIRE(p.filter_lambda >= 0.0, HDCG_ERR_ARG, "the filter's shifts lambda + i eps must be >= 0");
  HDCG_REQUIRE(p.surface_depth >= 0, HDCG_ERR_ARG, "surface depth must be >= 0");
}

// Level-1 subspace by the rational filter: wall noise, prod_i (H + lam + i eps)^-1
// by one multi-shift solve per vector, surface truncation, block Gram-Schmidt.
void build_subspace_rational(Ctx& c, const hdcg_subspace_params& p) {
  HDCG_REQUIRE(c.have_gauge && c.have_dwf, HDCG_ERR_STATE, "gauge field and DWF parameters required");
  check_filter(p);
  for (int mu = 0; mu < 4; ++mu)
    HDCG_REQUIRE(p.block[mu] >= 4, HDCG_ERR_ARG, "block extents must be >= 4 (Sec. 5.1)");
  if (!c.sub) c.sub = new Subspace();
  Subspace& s = *c.sub;
  const bool round_at_end = p.prec == HDCG_F16;
  subspace_init(c, s, p.block, p.nvec, round_at_end ? HDCG_F32 : p.prec);
  const int wp = s.prec == HDCG_F64 ? HDCG_F64 : HDCG_F32;
  std::vector<double> sig, cw;
  rational_filter_shifts(p.filter_lambda, p.filter_eps, p.filter_order, sig, cw);
  const int ns = p.filter_order;
  const size_t fb = c.field_bytes(wp);
  DevMem xs, ps, work, dscal;
  xs.ensure(fb * ns);
  ps.ensure(fb * ns);
  work.ensure(fb * 4);
  dscal.ensure(sizeof(double));
  const size_t fs = fb / 16;
  uint4* eta = work.as<uint4>();
  uint4* r = eta + fs;
  uint4* pb = r + fs;
  uint4* w = pb + fs;
  const unsigned g = (unsigned)((c.n5 + 255) / 256);
  ShiftCoef cc{};
  for (int i = 0; i < ns; ++i) cc.a[i] = cw[i];
  for (int k = 0; k < s.nvec; ++k) {
    DISPATCH_HI(wp, S, {
      k_wall_noise<S><<<g, 256, 0, c.stream>>>(eta, c.n5, c.lslog2, c.Ls, k, p.seed);
      HDCG_CUDA(cudaGetLastError());
      msh_filter<S>(c, wp, eta, xs.as<uint4>(), ps.as<uint4>(), r, pb, w, sig, p.inv_tol, p.inv_maxiter,
                    dscal.as<double>());
      k_msh_combine<S, S><<<g, 256, 0, c.stream>>>(xs.as<uint4>(), fs, ns, cc, s.vec(c, k), c.n5, c.Ls, 0);
    });
    HDCG_CUDA(cudaGetLastError());
    c.launches += 2;
  }
  truncate_surface(c, s, p.surface_depth);
  block_orthonormalise(c, s);
  if (round_at_end) round_to_f16(c, s);
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
}

// inv_steps steps of (H + inv_shift)^-1 applied to the current subspace, each
// followed by block Gram-Schmidt; then the surface truncation
void continue_subspace(Ctx& c, const hdcg_subspace_params& p) {
  HDCG_REQUIRE(c.sub && c.sub->nvec > 0, HDCG_ERR_STATE, "no subspace to continue from");
  HDCG_REQUIRE(p.surface_depth >= 0, HDCG_ERR_ARG, "surface depth must be >= 0");
  Subspace& s = *c.sub;
  const bool round_at_end = s.prec == HDCG_F16;
  if (round_at_end) {
    DevMem v16;
    std::swap(v16.p, s.vecs.p);
    std::swap(v16.bytes, s.vecs.bytes);
    s.prec = HDCG_F32;
    s.vecs.ensure((size_t)s.nvec * s.vec_bytes(c));
    convert_field(c, v16.as<uint4>(), HDCG_F16, s.vecs.as<uint4>(), HDCG_F32, s.nvec);
  }
  const int wp = s.prec == HDCG_F64 ? HDCG_F64 : HDCG_F32;
  for (int step = 0; step < p.inv_steps; ++step) {
    for (int k = 0; k < s.nvec; ++k) inverse_step(c, wp, s.vec(c, k), s.prec, p.inv_shift, p.inv_tol, p.inv_maxiter);
    block_orthonormalise(c, s);
  }
  truncate_surface(c, s, p.surface_depth);
  block_orthonormalise(c, s);
  if (round_at_end) round_to_f16(c, s);
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
}

// the level-1 subspace of src (same 4D lattice, fifth extent Ls1 <= Ls) promoted
// into this handle's Ls (k_promote), stored in prec and block-orthonormalised
void promote_subspace(Ctx& c, Ctx& src, int prec) {
  HDCG_REQUIRE(src.sub && src.sub->nvec > 0, HDCG_ERR_STATE, "the source handle has no subspace");
  HDCG_REQUIRE(&src != &c, HDCG_ERR_ARG, "promote from another handle");
  HDCG_REQUIRE(src.n5 / src.Ls == c.n5 / c.Ls, HDCG_ERR_ARG, "the handles' 4D lattices differ");
  for (int mu = 0; mu < 4; ++mu)
    HDCG_REQUIRE(src.dims[mu] == c.dims[mu], HDCG_ERR_ARG, "the handles' 4D lattices differ");
  HDCG_REQUIRE(src.Ls <= c.Ls, HDCG_ERR_ARG, "the source's fifth extent must not exceed Ls");
  HDCG_REQUIRE(prec == HDCG_F64 || prec == HDCG_F32 || prec == HDCG_F16, HDCG_ERR_ARG,
               "subspace precision must be F64, F32 or F16");
  HDCG_CUDA(cudaStreamSynchronize(src.stream));
  const Subspace& s1 = *src.sub;
  if (!c.sub) c.sub = new Subspace();
  Subspace& s = *c.sub;
  const bool round_at_end = prec == HDCG_F16;
  subspace_init(c, s, s1.block, s1.nvec, round_at_end ? HDCG_F32 : prec);
  const size_t n = c.n5 * s.nvec;
  DISPATCH_SUB(s1.prec, Si, {
    DISPATCH_SUB(s.prec, So, {
      k_promote<Si, So><<<(unsigned)((n + 255) / 256), 256, 0, c.stream>>>(
          s1.vecs.as<uint4>(), src.n5, src.Ls, s.vecs.as<uint4>(), c.n5, c.Ls, c.lslog2, s.nvec);
    });
  });
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
  block_orthonormalise(c, s);
  if (round_at_end) round_to_f16(c, s);
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
}

}  // namespace hdcg
