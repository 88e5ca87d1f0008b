// The generalised preconditioned CG and its family of preconditioners
// (Sec. 4.5, Fig. pcg_general, Tables precs and algos, Table preconditioner).
//
// Fig. pcg_general: x_0 = V_start, r_0 = b - H x_0, y_0 = M_1 r_0,
// p_0 = M_2 y_0; per iteration w = M_3 H p, alpha = (r, y) / (p, w),
// x += alpha p, r -= alpha w, y = M_1 r, beta = (r_new, y_new) / (r, y) (or the
// flexible form), p = M_2 y + beta p; x = V_end.  Table algos fills the slots
// from Q = P A^-1 R, P_L = 1 - H Q, P_R = 1 - Q H and a smoother M:
//   PREC    M_1 = M
//   AD      M_1 = M + Q
//   DEF1    M_1 = M, M_3 = P_L, r_0 projected by P_L, V_end = Q b + P_R x
//   DEF2    M_1 = M, M_2 = P_R, V_start = Q b + P_R x
//   A-DEF1  M_1 = M P_L + Q
//   A-DEF2  M_1 = P_R M + Q, V_start = Q b + P_R x
//   BNN     M_1 = P_R M P_L + Q (from x, or from the DEF2 start)
//   V(1,1)  M_1 = M P_L + P_R M + Q - M P_L H M (the symmetric two-grid cycle)
//   MssDef  A-DEF2 with M = 1
// Readings: DEF1 iterates on the deflated system P_L H x = P_L b, so its start
// residual is projected; A-DEF1 has M_2 = 1.
// Smoothers (Table preconditioner): M_IRS (CG on H + lambda from zero, a fixed
// number of iterations), M_IRSpoly (the same CG's alpha_k, beta_k frozen from
// one pass on the right-hand side b and replayed: a fixed polynomial in H),
// the Chebyshev-acceleration polynomial of H on [lo, hi], or none.
//
// One right-hand side at a time, every field and every operator in one
// working precision (FP64 or FP32); scalars on the host.  This is the study
// solver of the family; the production A-DEF2 path is solver.cu.
#include <cmath>
#include <vector>

#include "coarse.cuh"

namespace hdcg {

namespace {

struct Family {
  Ctx& c;
  const hdcg_params& prm;
  hdcg_stats* st;
  int wp;
  std::vector<DevMem> pool;
  int top = 0;
  DevMem scal, cv;
  std::vector<double> poly_a, poly_b;   // M_IRSpoly coefficients

  Family(Ctx& c_, const hdcg_params& p, hdcg_stats* s, int wp_) : c(c_), prm(p), st(s), wp(wp_), pool(24) {
    scal.ensure(4 * sizeof(double));
  }
  // work fields, handed out and returned in stack order
  uint4* get() {
    HDCG_REQUIRE(top < (int)pool.size(), HDCG_ERR_STATE, "family solver: out of work fields");
    pool[top].ensure(c.field_bytes(wp));
    return pool[top++].as<uint4>();
  }
  void put(int n) { top -= n; }

  double dot(const uint4* a, const uint4* b) {
    redot2(c, wp, a, b, nullptr, scal.as<double>());
    double h[2];
    HDCG_CUDA(cudaMemcpyAsync(h, scal.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    HDCG_CUDA(cudaStreamSynchronize(c.stream));
    return h[0];
  }
  double nrm2(const uint4* a) {
    norm2(c, a, wp, 0, scal.as<double>());
    double h = 0;
    HDCG_CUDA(cudaMemcpyAsync(&h, scal.p, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    HDCG_CUDA(cudaStreamSynchronize(c.stream));
    return h;
  }
  void copy(const uint4* in, uint4* out) {
    if (in != out) HDCG_CUDA(cudaMemcpyAsync(out, in, c.field_bytes(wp), cudaMemcpyDeviceToDevice, c.stream));
  }
  // y = a x + b y
  void axpy(double a, const uint4* x, double b, uint4* y) { axpby(c, a, wp, x, b, wp, y); }

  void H(const uint4* in, uint4* out) {
    apply_mdagm(c, wp, in, out, nullptr);
    if (st) ++st->n_mdagm_outer;
  }
  // out = Q in = P A^-1 R in
  void Q(const uint4* in, uint4* out) {
    Subspace& s = *c.sub;
    Coarse& A = *c.coarse;
    const int cp = A.vec_prec();
    const size_t nc = A.Vc * A.nvec;
    cv.ensure(2 * nc * 16);
    char* cin = cv.as<char>();
    char* cout = cin + nc * 16;
    restrict_field(c, s, in, wp, cin, cp);
    const int it = coarse_cg(c, A, cin, cout, prm.coarse_tol, prm.coarse_maxiter);
    if (st) {
      st->coarse_iterations += it;
      if (it > st->coarse_iterations_max) st->coarse_iterations_max = it;
    }
    prolong_field(c, s, cout, cp, out, wp, nullptr);
  }
  // out = P_L in = in - H Q in
  void PL(const uint4* in, uint4* out) {
    uint4* t = get();
    Q(in, t);
    H(t, out);
    axpy(1.0, in, -1.0, out);
    put(1);
  }
  // out = P_R in = in - Q H in
  void PR(const uint4* in, uint4* out) {
    uint4* t = get();
    H(in, t);
    Q(t, out);
    axpy(1.0, in, -1.0, out);
    put(1);
  }

  // CG on H + lambda from zero: n iterations; record (alpha_k, beta_k) if asked
  void mirs(const uint4* in, uint4* out, std::vector<double>* ra, std::vector<double>* rb) {
    const double lam = prm.mirs_shift;
    uint4* r = get();
    uint4* p = get();
    uint4* w = get();
    HDCG_CUDA(cudaMemsetAsync(out, 0, c.field_bytes(wp), c.stream));
    copy(in, r);
    copy(in, p);
    double rr = nrm2(r);
    for (int k = 0; k < prm.mirs_iter && rr > 0.0; ++k) {
      apply_mdagm(c, wp, p, w, nullptr, 1.0, lam, p);
      if (st) ++st->n_mdagm_sloppy;
      const double pw = dot(p, w);
      HDCG_REQUIRE(std::isfinite(pw) && pw > 0.0, HDCG_ERR_BREAKDOWN, "M_IRS: (p, (H + lambda) p) <= 0");
      const double al = rr / pw;
      axpy(al, p, 1.0, out);
      axpy(-al, w, 1.0, r);
      const double rn = nrm2(r);
      const double be = rn / rr;
      if (ra) ra->push_back(al);
      if (rb) rb->push_back(be);
      axpy(1.0, r, be, p);
      rr = rn;
    }
    put(3);
  }
  // the frozen polynomial: the same recurrences with the recorded coefficients
  void mirs_poly(const uint4* in, uint4* out) {
    const double lam = prm.mirs_shift;
    uint4* r = get();
    uint4* p = get();
    uint4* w = get();
    HDCG_CUDA(cudaMemsetAsync(out, 0, c.field_bytes(wp), c.stream));
    copy(in, r);
    copy(in, p);
    for (size_t k = 0; k < poly_a.size(); ++k) {
      axpy(poly_a[k], p, 1.0, out);
      apply_mdagm(c, wp, p, w, nullptr, 1.0, lam, p);
      if (st) ++st->n_mdagm_sloppy;
      axpy(-poly_a[k], w, 1.0, r);
      axpy(1.0, r, poly_b[k], p);
    }
    put(3);
  }
  // Chebyshev acceleration: 1 - x p(x) = T_n((theta - x) / delta) / T_n(theta / delta)
  void cheb(const uint4* in, uint4* out) {
    const double lo = prm.cheb_lo, hi = prm.cheb_hi;
    const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
    double rho = 1.0 / sigma;
    uint4* s = get();
    uint4* d = get();
    uint4* hd = get();
    HDCG_CUDA(cudaMemsetAsync(out, 0, c.field_bytes(wp), c.stream));
    copy(in, s);
    HDCG_CUDA(cudaMemsetAsync(d, 0, c.field_bytes(wp), c.stream));
    axpy(1.0 / theta, in, 0.0, d);
    for (int k = 0; k < prm.cheb_order; ++k) {
      axpy(1.0, d, 1.0, out);
      if (k == prm.cheb_order - 1) break;
      apply_mdagm(c, wp, d, hd, nullptr);
      if (st) ++st->n_mdagm_sloppy;
      axpy(-1.0, hd, 1.0, s);
      const double rn = 1.0 / (2.0 * sigma - rho);
      axpy(2.0 * rn / delta, s, rn * rho, d);
      rho = rn;
    }
    put(3);
  }
  void M(const uint4* in, uint4* out) {
    switch (prm.smoother) {
      case HDCG_SMOOTHER_MIRS: mirs(in, out, nullptr, nullptr); break;
      case HDCG_SMOOTHER_MIRSPOLY: mirs_poly(in, out); break;
      case HDCG_SMOOTHER_CHEBYSHEV: cheb(in, out); break;
      default: copy(in, out); break;
    }
  }

  // out = M_1 r
  void M1(int alg, const uint4* r, uint4* out) {
    switch (alg) {
      case HDCG_ALG_PREC:
      case HDCG_ALG_DEF1:
      case HDCG_ALG_DEF2: M(r, out); break;
      case HDCG_ALG_AD: {
        uint4* q = get();
        M(r, out);
        Q(r, q);
        axpy(1.0, q, 1.0, out);
        put(1);
        break;
      }
      case HDCG_ALG_ADEF1: {
        uint4* t = get();
        uint4* q = get();
        PL(r, t);
        M(t, out);
        Q(r, q);
        axpy(1.0, q, 1.0, out);
        put(2);
        break;
      }
      case HDCG_ALG_ADEF2_FAMILY:
      case HDCG_ALG_MSSDEF: {
        uint4* t = get();
        uint4* q = get();
        if (alg == HDCG_ALG_MSSDEF) copy(r, t);
        else M(r, t);
        PR(t, out);
        Q(r, q);
        axpy(1.0, q, 1.0, out);
        put(2);
        break;
      }
      case HDCG_ALG_BNN:
      case HDCG_ALG_BNN_DEF2START: {
        uint4* t = get();
        uint4* u = get();
        PL(r, t);
        M(t, u);
        PR(u, out);
        Q(r, t);
        axpy(1.0, t, 1.0, out);
        put(2);
        break;
      }
      case HDCG_ALG_V11: {
        uint4* mr = get();
        uint4* t = get();
        uint4* u = get();
        M(r, mr);
        PL(r, t);
        M(t, out);             // M P_L r
        PR(mr, u);
        axpy(1.0, u, 1.0, out);  // + P_R M r
        Q(r, u);
        axpy(1.0, u, 1.0, out);  // + Q r
        H(mr, t);
        PL(t, u);
        M(u, t);
        axpy(-1.0, t, 1.0, out);  // - M P_L H M r
        put(3);
        break;
      }
      default: throw Error{HDCG_ERR_ARG, "unknown algorithm"};
    }
  }
};

bool def2_start(int alg) {
  return alg == HDCG_ALG_DEF2 || alg == HDCG_ALG_ADEF2_FAMILY || alg == HDCG_ALG_BNN_DEF2START ||
         alg == HDCG_ALG_MSSDEF;
}

bool needs_coarse(int alg) { return alg != HDCG_ALG_PREC; }

}  // namespace

bool is_family_algorithm(int alg) { return alg >= HDCG_ALG_PREC && alg <= HDCG_ALG_ADEF2_FAMILY; }

// One right-hand side: b64, x64 internal FP64 fields.  Stops when the
// recursive residual reaches tol relative to |b| (DEF1: the projected one);
// the true residual |b - H x| / |b| of V_end is recomputed in FP64.
int solve_family(Ctx& c, const uint4* b64, uint4* x64, double tol, const hdcg_params& prm, hdcg_stats* st) {
  const int alg = prm.algorithm;
  const int wp = prm.outer_prec;
  HDCG_REQUIRE(wp == HDCG_F64 || wp == HDCG_F32, HDCG_ERR_ARG, "the family solves run in F64 or F32");
  if (needs_coarse(alg)) HDCG_REQUIRE(c.sub && c.coarse, HDCG_ERR_STATE, "deflation needs a subspace and A");
  HDCG_REQUIRE(prm.smoother >= HDCG_SMOOTHER_MIRS && prm.smoother <= HDCG_SMOOTHER_NONE, HDCG_ERR_ARG,
               "unknown smoother");
  if (prm.smoother == HDCG_SMOOTHER_CHEBYSHEV)
    HDCG_REQUIRE(prm.cheb_order >= 1 && prm.cheb_lo > 0 && prm.cheb_hi > prm.cheb_lo, HDCG_ERR_ARG,
                 "Chebyshev smoother needs order >= 1 and 0 < lo < hi");
  Family f(c, prm, st, wp);
  uint4* b = f.get();
  uint4* x = f.get();
  uint4* r = f.get();
  uint4* y = f.get();
  uint4* p = f.get();
  uint4* w = f.get();
  convert_field(c, b64, HDCG_F64, b, wp);
  const double bb = f.nrm2(b);
  HDCG_CUDA(cudaMemsetAsync(x64, 0, c.field_bytes(HDCG_F64), c.stream));
  if (bb == 0.0) {
    HDCG_CUDA(cudaStreamSynchronize(c.stream));
    return HDCG_OK;
  }
  if (prm.smoother == HDCG_SMOOTHER_MIRSPOLY) f.mirs(b, w, &f.poly_a, &f.poly_b);  // coefficients from b
  // V_start
  if (def2_start(alg)) {
    f.Q(b, x);          // Q b + P_R 0
  } else {
    HDCG_CUDA(cudaMemsetAsync(x, 0, c.field_bytes(wp), c.stream));
  }
  f.H(x, r);
  f.axpy(1.0, b, -1.0, r);  // r = b - H x
  if (alg == HDCG_ALG_DEF1) {
    f.PL(r, w);
    f.copy(w, r);
  }
  f.M1(alg, r, y);
  if (alg == HDCG_ALG_DEF2) f.PR(y, p);
  else f.copy(y, p);
  double ry = f.dot(r, y);
  double rr = f.nrm2(r);
  int it = 0;
  uint4* yn = f.get();
  while (it < prm.maxiter && rr > tol * tol * bb) {
    f.H(p, w);
    if (alg == HDCG_ALG_DEF1) {
      uint4* t = f.get();
      f.PL(w, t);
      f.copy(t, w);
      f.put(1);
    }
    const double pw = f.dot(p, w);
    HDCG_REQUIRE(std::isfinite(pw) && pw > 0.0, HDCG_ERR_BREAKDOWN, "(p, M3 H p) <= 0");
    const double alpha = ry / pw;
    f.axpy(alpha, p, 1.0, x);
    f.axpy(-alpha, w, 1.0, r);
    ++it;
    rr = f.nrm2(r);
    HDCG_REQUIRE(std::isfinite(rr), HDCG_ERR_NONFINITE, "non-finite residual");
    if (rr <= tol * tol * bb) break;
    f.M1(alg, r, yn);
    const double ryn = f.dot(r, yn);
    const double beta = prm.flexible ? (ryn - f.dot(r, y)) / ry : ryn / ry;
    if (alg == HDCG_ALG_DEF2) {
      uint4* t = f.get();
      f.PR(yn, t);
      f.axpy(1.0, t, beta, p);
      f.put(1);
    } else {
      f.axpy(1.0, yn, beta, p);
    }
    f.copy(yn, y);
    ry = ryn;
  }
  // V_end
  if (alg == HDCG_ALG_DEF1) {
    f.PR(x, w);
    f.Q(b, y);
    f.axpy(1.0, y, 1.0, w);
    f.copy(w, x);
  }
  convert_field(c, x, wp, x64, HDCG_F64);
  // true residual in FP64
  uint4* r64 = c.scratch(HDCG_F64, 17);
  apply_mdagm(c, HDCG_F64, x64, r64, nullptr, -1.0, 1.0, b64);
  if (st) ++st->n_mdagm_f64;
  norm2(c, r64, HDCG_F64, 0, f.scal.as<double>());
  double tr = 0;
  HDCG_CUDA(cudaMemcpyAsync(&tr, f.scal.p, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
  if (st) {
    st->iterations += it;
    st->true_residual = std::max(st->true_residual, std::sqrt(tr / bb));
  }
  return rr <= tol * tol * bb ? HDCG_OK : HDCG_NOT_CONVERGED;
}

}  // namespace hdcg
