// Krylov solvers of the HDCG library (Boyle, arXiv 1402.2585).
//
//  * cg_fixed / cg_to_tol: CG on (H + shift) in one storage precision; with a
//    fixed iteration count and zero start this is the infra-red shifted
//    smoother M_IRS(H, N, lambda) of Sec. 4.3.
//  * apply_M1: the A-DEF2 preconditioner M1 = P_R M_IRS + Q of Table algos,
//    evaluated as y = z + Q (r - H z), z = M_IRS r (P_R = 1 - Q H), with
//    Q = P A^-1 R (Sec. 2) and the coarse CG stopped at a relative residual
//    (Table optimised: 0.04).
//  * solve_one: the generalised preconditioned CG of Fig. pcg_general with the
//    A-DEF2 row (V_start = Q b, M2 = M3 = 1) or plain CG (M1 = 1).  Flexible
//    beta is the Polak-Ribiere form (r_{k+1}, y_{k+1} - y_k) / (r_k, y_k)
//    (reading of the flexible CG the paper cites).  The outer recursion runs
//    in the outer precision; the solution accumulates in FP64 and the true
//    residual b - H x is recomputed with the FP64 operator whenever |r| has
//    fallen by reliable_delta, and at convergence (reliable updates).
// All inner products are FP64 device scalars; alpha and beta are formed on
// the device.  The host reads two scalars per outer iteration to decide on
// reliable updates and termination.
#include <chrono>
#include <cmath>
#include <cstring>

#include "coarse.cuh"

namespace hdcg {

// scratch slot roles (per precision): see header comment of this file
enum {
  SL_XLO = 3, SL_R = 4, SL_P = 5, SL_W = 6, SL_Y = 7, SL_YN = 8,
  SL_RS = 9, SL_Z = 10, SL_MRES = 11, SL_MP = 12, SL_MW = 13, SL_T = 14,
  SL_XHI = 15, SL_B = 16, SL_R64 = 17, SL_CGB = 18, SL_CGX = 19
};
// device scalar slots (doubles)
enum {
  D_PW = 0, D_RR = 1, D_RY = 2, D_RYN = 3 /* 2 */, D_BB = 6, D_TMP = 7, D_NREAL = 8,
  D_MRR = 16 /* 2 */, D_MPW = 18, D_MPP = 19, D_CRR = 24 /* 2 */, D_CPW = 26, D_CPP = 27,
  D_RYO = 30 /* 2 */, D_AMAX = 32 /* unsigned */
};

// 16-bit preconditioner input: unit RMS per real, unless that puts a real
// beyond SCALED_PEAK (a localised residual, e.g. of a point source, whose
// peak is up to sqrt(#reals) times its RMS): then the peak is SCALED_PEAK.
// The sloppy H multiplies magnitudes by up to ~10^2, so FP16's 65504 is not
// reached, and reals down to 1e-6 of the peak stay normal FP16 numbers.
constexpr double SCALED_PEAK = 64.0;

static double* dsc(Ctx& c, int slot) { return c.scalars.as<double>() + slot * RMAX; }

// read scalar slots [slot, slot + n) of right-hand side 0
static void read_scalars(Ctx& c, int slot, int n, double* h) {
  for (int i = 0; i < n; ++i)
    HDCG_CUDA(cudaMemcpyAsync(h + i, dsc(c, slot + i), sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
}

static void copy_scalar(Ctx& c, int dst, int src) {
  HDCG_CUDA(cudaMemcpyAsync(dsc(c, dst), dsc(c, src), sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
}

static void copy_field(Ctx& c, int prec, const uint4* in, uint4* out) {
  HDCG_CUDA(cudaMemcpyAsync(out, in, c.field_bytes(prec), cudaMemcpyDeviceToDevice, c.stream));
}

// ---------------------------------------------------------------------------
// CG on (H + shift) in one precision, zero start.
// niter_fixed > 0: exactly that many iterations (M_IRS); otherwise iterate to
// |r| <= tol |b| (checked on the host every iteration).
// ---------------------------------------------------------------------------
static void copy_fields(Ctx& c, int prec, const uint4* in, uint4* out, int R) {
  HDCG_CUDA(cudaMemcpyAsync(out, in, c.field_bytes(prec) * R, cudaMemcpyDeviceToDevice, c.stream));
}

static void copy_scalars(Ctx& c, int dst, int src, int R) {
  HDCG_CUDA(cudaMemcpyAsync(dsc(c, dst), dsc(c, src), R * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
}

static int cg_shifted(Ctx& c, int prec, const uint4* b, uint4* x, double shift, int niter_fixed, double tol,
                      int maxiter, int* n_mdagm, int R = 1) {
  HDCG_REQUIRE(R == 1 || niter_fixed > 0, HDCG_ERR_ARG, "several right-hand sides need a fixed iteration count");
  uint4* res = c.scratch(prec, SL_MRES, R);
  uint4* p = c.scratch(prec, SL_MP, R);
  zero_field(c, x, prec, R);
  copy_fields(c, prec, b, res, R);
  copy_fields(c, prec, b, p, R);
  norm2(c, b, prec, 0, dsc(c, D_MRR), R);
  copy_scalars(c, D_MPP, D_MRR, R);
  double bb = 0.0;
  if (niter_fixed <= 0) {
    read_scalars(c, D_MRR, 1, &bb);
    if (bb == 0.0) return 0;
  }
  const int nit = niter_fixed > 0 ? niter_fixed : maxiter;
  int it = 0;
  for (; it < nit; ++it) {
    const int par = it & 1;
    apply_mdagm_cg(c, prec, p, shift, x, res, dsc(c, D_MRR + par), dsc(c, D_MPW), dsc(c, D_MPP),
                   dsc(c, D_MRR + (par ^ 1)), R);
    if (n_mdagm) *n_mdagm += R;
    if (niter_fixed <= 0) {
      double rr = 0.0;
      read_scalars(c, D_MRR + (par ^ 1), 1, &rr);
      HDCG_REQUIRE(std::isfinite(rr), HDCG_ERR_NONFINITE, "non-finite residual in CG");
      if (rr <= tol * tol * bb) {
        ++it;
        break;
      }
    } else if (it == nit - 1) {
      break;
    }
    ScalarRef be;
    be.num = dsc(c, D_MRR + (par ^ 1));
    be.den0 = dsc(c, D_MRR + par);
    update_p(c, prec, p, res, be, dsc(c, D_MPP), R);
  }
  return niter_fixed > 0 ? nit : it;
}

// ---------------------------------------------------------------------------
// Q t = P A^-1 R t (+ add) in the sloppy precision
// ---------------------------------------------------------------------------
// out (precision oprec) = add (oprec) + P A^-1 R t, t in precision sp
static void apply_Q(Ctx& c, int sp, const uint4* t, uint4* out, int oprec, const uint4* add, const hdcg_params& prm,
                    hdcg_stats* st) {
  Subspace& s = *c.sub;
  Coarse& A = *c.coarse;
  const int cp = A.vec_prec();
  const size_t nc = A.Vc * A.nvec;
  A.qvec.ensure(2 * nc * 16);
  char* q0 = A.qvec.as<char>();
  void* cin = q0;
  void* cout = q0 + nc * 16;
  {
    PhaseTimer pt(c, PH_TRANSFER);
    restrict_field(c, s, t, sp, cin, cp);
  }
  int it = 0;
  {
    PhaseTimer pt(c, PH_COARSE);
    it = coarse_cg(c, A, cin, cout, prm.coarse_tol, prm.coarse_maxiter);
  }
  if (st) {
    st->coarse_iterations += it;
    if (it > st->coarse_iterations_max) st->coarse_iterations_max = it;
  }
  PhaseTimer pt(c, PH_TRANSFER);
  prolong_field(c, s, cout, cp, out, oprec, add);
}

// y = M1 r in precision op (A-DEF2) ; r in op.  M1 is linear (M_IRS runs a
// fixed number of CG steps from zero; Q is linear), so a 16-bit preconditioner
// runs on r scaled to unit RMS per real (keeping residual entries inside the
// normal FP16 range) and its result is scaled back.
static void apply_M1(Ctx& c, int op, int sp, const uint4* r, uint4* y, const hdcg_params& prm, hdcg_stats* st) {
  const uint4* rs = r;
  const bool scaled = is_16bit(sp);
  if (scaled) {
    norm2(c, r, op, 0, dsc(c, D_TMP));
    cap_scale(c, r, op, dsc(c, D_NREAL), dsc(c, D_TMP), SCALED_PEAK, reinterpret_cast<unsigned*>(dsc(c, D_AMAX)));
    uint4* t = c.scratch(sp, SL_RS);
    convert_scaled(c, r, op, t, sp, dsc(c, D_NREAL), dsc(c, D_TMP), 0);
    rs = t;
  } else if (sp != op) {
    uint4* t = c.scratch(sp, SL_RS);
    convert_field(c, r, op, t, sp);
    rs = t;
  }
  if (prm.sloppy_codec) {
    HDCG_REQUIRE(scaled, HDCG_ERR_ARG, "sloppy_codec needs a 16-bit sloppy precision (unit-RMS input)");
    codec_roundtrip(c, const_cast<uint4*>(rs), sp, prm.sloppy_codec);
  }
  uint4* z = c.scratch(sp, SL_Z);
  uint4* t = c.scratch(sp, SL_T);
  int nm = 0;
  {
    PhaseTimer pt(c, PH_H_SLOPPY);
    cg_shifted(c, sp, rs, z, prm.mirs_shift, prm.mirs_iter, 0.0, prm.mirs_iter, &nm);
    apply_mdagm(c, sp, z, t, nullptr, -1.0, 1.0, rs);  // t = r - H z
    ++nm;
  }
  if (st) st->n_mdagm_sloppy += nm;
  if (sp == op) {
    apply_Q(c, sp, t, y, sp, z, prm, st);
  } else if (scaled) {
    // the coarse-grid correction amplifies low modes by up to 1 / lambda_min(H),
    // beyond the FP16 range: z + Q t is formed and kept in FP32
    uint4* zf = c.scratch(HDCG_F32, SL_Z);
    uint4* yf = c.scratch(HDCG_F32, SL_MRES);
    convert_field(c, z, sp, zf, HDCG_F32);
    apply_Q(c, sp, t, yf, HDCG_F32, zf, prm, st);
    convert_scaled(c, yf, HDCG_F32, y, op, dsc(c, D_NREAL), dsc(c, D_TMP), 1);
  } else {
    uint4* ys = c.scratch(sp, SL_MRES);
    apply_Q(c, sp, t, ys, sp, z, prm, st);
    convert_field(c, ys, sp, y, op);
  }
}

// x_hi (FP64) = Q b  (16-bit: on b scaled to unit RMS, scaled back)
static void start_vector(Ctx& c, int sp, const uint4* b64, uint4* xhi, const hdcg_params& prm, hdcg_stats* st) {
  uint4* bs = c.scratch(sp, SL_RS);
  const bool scaled = is_16bit(sp);
  if (scaled) {
    norm2(c, b64, HDCG_F64, 0, dsc(c, D_TMP));
    cap_scale(c, b64, HDCG_F64, dsc(c, D_NREAL), dsc(c, D_TMP), SCALED_PEAK,
              reinterpret_cast<unsigned*>(dsc(c, D_AMAX)));
    convert_scaled(c, b64, HDCG_F64, bs, sp, dsc(c, D_NREAL), dsc(c, D_TMP), 0);
  } else {
    convert_field(c, b64, HDCG_F64, bs, sp);
  }
  if (scaled) {
    uint4* x0 = c.scratch(HDCG_F32, SL_T);
    apply_Q(c, sp, bs, x0, HDCG_F32, nullptr, prm, st);
    convert_scaled(c, x0, HDCG_F32, xhi, HDCG_F64, dsc(c, D_NREAL), dsc(c, D_TMP), 1);
  } else {
    uint4* x0 = c.scratch(sp, SL_T);
    apply_Q(c, sp, bs, x0, sp, nullptr, prm, st);
    convert_field(c, x0, sp, xhi, HDCG_F64);
  }
}

// r64 = b64 - H x64 for one right-hand side with the double-float operator (FP64
// accuracy on the FP32 units): x and b enter as double-float copies, r leaves as
// FP64.  Several right-hand sides run one after another, so the double-float
// work fields are one field each whatever the batch.
static void residual_df(Ctx& c, const uint4* b64, const uint4* x64, uint4* r64) {
  uint4* xd = c.scratch(HDCG_DF64, 5);
  uint4* bd = c.scratch(HDCG_DF64, 6);
  uint4* rd = c.scratch(HDCG_DF64, 7);
  convert_field(c, x64, HDCG_F64, xd, HDCG_DF64);
  convert_field(c, b64, HDCG_F64, bd, HDCG_DF64);
  apply_mdagm(c, HDCG_DF64, xd, rd, nullptr, -1.0, 1.0, bd);
  convert_field(c, rd, HDCG_DF64, r64, HDCG_F64);
}

static double true_residual(Ctx& c, int op, const uint4* b64, const uint4* xhi, uint4* r, hdcg_stats* st) {
  uint4* r64 = c.scratch(HDCG_F64, SL_R64);
  {
    PhaseTimer pt(c, PH_H_F64);
    residual_df(c, b64, xhi, r64);
  }
  if (st) ++st->n_mdagm_f64;
  norm2(c, r64, HDCG_F64, 0, dsc(c, D_RR));
  if (op != HDCG_F64) convert_field(c, r64, HDCG_F64, r, op);
  else copy_field(c, HDCG_F64, r64, r);
  double rr = 0.0;
  read_scalars(c, D_RR, 1, &rr);
  return rr;
}

// one right-hand side: b64, x64 internal FP64 fields
static int solve_one(Ctx& c, const uint4* b64, uint4* x64, double tol, const hdcg_params& prm, hdcg_stats* st) {
  const int op = prm.outer_prec, sp = prm.sloppy_prec;
  const bool adef2 = prm.algorithm == HDCG_ALG_ADEF2;
  HDCG_REQUIRE(op == HDCG_F64 || op == HDCG_F32, HDCG_ERR_ARG, "outer precision must be F64 or F32");
  if (adef2) {
    HDCG_REQUIRE(c.sub && c.coarse, HDCG_ERR_STATE, "A-DEF2 needs a subspace and a coarse operator");
    HDCG_REQUIRE(sp >= HDCG_F64 && sp <= HDCG_BF16T, HDCG_ERR_ARG, "bad sloppy precision");
  }
  uint4* xlo = c.scratch(op, SL_XLO);
  uint4* r = c.scratch(op, SL_R);
  uint4* p = c.scratch(op, SL_P);
  uint4* y = c.scratch(op, SL_Y);
  uint4* yn = c.scratch(op, SL_YN);
  uint4* xhi = x64;

  {
    const double nreal = (double)c.n5 * 24.0;
    HDCG_CUDA(cudaMemcpyAsync(dsc(c, D_NREAL), &nreal, sizeof(double), cudaMemcpyHostToDevice, c.stream));
    HDCG_CUDA(cudaStreamSynchronize(c.stream));
  }
  norm2(c, b64, HDCG_F64, 0, dsc(c, D_BB));
  double bb = 0.0;
  read_scalars(c, D_BB, 1, &bb);
  zero_field(c, xhi, HDCG_F64);
  zero_field(c, xlo, op);
  if (bb == 0.0) {
    st->true_residual = 0.0;
    return HDCG_OK;
  }
  const double stop = tol * tol * bb;
  if (adef2) start_vector(c, sp, b64, xhi, prm, st);
  double rr = true_residual(c, op, b64, xhi, r, st);
  double rr_rel = rr;
  if (rr <= stop) {
    st->true_residual = std::sqrt(rr / bb);
    return HDCG_OK;
  }
  // y_0 = M1 r_0, p_0 = y_0, ry = (r, y)
  if (adef2) {
    apply_M1(c, op, sp, r, y, prm, st);
    copy_field(c, op, y, p);
    redot2(c, op, r, y, nullptr, dsc(c, D_RYN));
    copy_scalar(c, D_RY, D_RYN);
  } else {
    copy_field(c, op, r, p);
    copy_scalar(c, D_RY, D_RR);
  }
  int it = 0;
  int status = HDCG_NOT_CONVERGED;
  while (it < prm.maxiter) {
    {
      PhaseTimer pt(c, PH_H_OUTER);
      apply_mdagm_cg(c, op, p, 0.0, xlo, r, dsc(c, D_RY), dsc(c, D_PW), nullptr, dsc(c, D_RR));
    }
    ++st->n_mdagm_outer;
    ++it;
    double h[2];
    read_scalars(c, D_PW, 2, h);  // pw, rr
    HDCG_REQUIRE(std::isfinite(h[0]) && std::isfinite(h[1]), HDCG_ERR_NONFINITE, "non-finite residual");
    HDCG_REQUIRE(h[0] > 0.0, HDCG_ERR_BREAKDOWN, "(p, Hp) <= 0");
    rr = h[1];
    if (rr <= prm.reliable_delta * prm.reliable_delta * rr_rel || rr <= stop || it >= prm.maxiter) {
      accum_hi(c, HDCG_F64, xhi, op, xlo);
      rr = true_residual(c, op, b64, xhi, r, st);
      rr_rel = rr;
      ++st->reliable_updates;
      if (rr <= stop) {
        status = HDCG_OK;
        break;
      }
    }
    if (adef2) {
      apply_M1(c, op, sp, r, yn, prm, st);
      redot2(c, op, r, yn, y, dsc(c, D_RYN));  // (r, y_new), (r, y_old)
      ScalarRef be;
      be.num = dsc(c, D_RYN);
      be.den0 = dsc(c, D_RY);
      be.den1 = prm.flexible ? dsc(c, D_RYN) + 1 : nullptr;  // (r, y_old): second value of the pair
      update_p(c, op, p, yn, be, nullptr);
      copy_scalar(c, D_RY, D_RYN);
      std::swap(y, yn);
    } else {
      ScalarRef be;
      be.num = dsc(c, D_RR);
      be.den0 = dsc(c, D_RY);
      update_p(c, op, p, r, be, nullptr);
      copy_scalar(c, D_RY, D_RR);
    }
  }
  st->iterations += it;
  const double tr = std::sqrt(rr / bb);
  if (tr > st->true_residual) st->true_residual = tr;
  return status;
}


// ---------------------------------------------------------------------------
// Several right-hand sides in lockstep (the batched driver).  Every kernel
// covers all R right-hand sides (grid y or a trailing right-hand-side index);
// alpha and beta are per right-hand side; a device mask freezes right-hand
// sides whose true residual has converged.  The coarse level reads the
// subspace and the little Dirac operator once per step for all of them.
// ---------------------------------------------------------------------------
static void apply_Q_multi(Ctx& c, int sp, int R, const uint4* t, uint4* out, int oprec, const uint4* add,
                          const hdcg_params& prm, hdcg_stats* st, int add_prec = -1,
                          const double* un_num = nullptr, const double* un_den = nullptr) {
  Subspace& s = *c.sub;
  Coarse& A = *c.coarse;
  const int cp = A.vec_prec();
  const size_t nc = A.Vc * A.nvec * (size_t)R;
  A.qvec.ensure(2 * nc * 16);
  char* q0 = A.qvec.as<char>();
  void* cin = q0;
  void* cout = q0 + nc * 16;
  {
    PhaseTimer pt(c, PH_TRANSFER);
    restrict_multi(c, s, t, sp, R, cin, cp);
  }
  int it = 0;
  {
    PhaseTimer pt(c, PH_COARSE);
    it = coarse_cg_multi(c, A, R, cin, cout, prm.coarse_tol, prm.coarse_maxiter);
  }
  if (st) {
    st->coarse_iterations += it;
    if (it > st->coarse_iterations_max) st->coarse_iterations_max = it;
  }
  PhaseTimer pt(c, PH_TRANSFER);
  prolong_multi(c, s, cout, cp, R, out, oprec, add, add_prec, un_num, un_den);
}

// y = M1 r for R right-hand sides.  Work fields: rs, z and the CG's residual and
// direction (sloppy precision); r - H z reuses the CG direction's slot.  A
// 16-bit preconditioner's output is prolonged straight into y in the outer
// precision, with z added from FP16 and the unit-RMS scaling undone there.
static void apply_M1_multi(Ctx& c, int op, int sp, int R, const uint4* r, uint4* y, const hdcg_params& prm,
                           hdcg_stats* st) {
  const uint4* rs = r;
  const bool scaled = is_16bit(sp);
  if (scaled) {
    norm2(c, r, op, 0, dsc(c, D_TMP), R);
    cap_scale(c, r, op, dsc(c, D_NREAL), dsc(c, D_TMP), SCALED_PEAK, reinterpret_cast<unsigned*>(dsc(c, D_AMAX)),
              R);
    uint4* t = c.scratch(sp, SL_RS, R);
    convert_scaled(c, r, op, t, sp, dsc(c, D_NREAL), dsc(c, D_TMP), 0, R);
    rs = t;
  } else if (sp != op) {
    uint4* t = c.scratch(sp, SL_RS, R);
    convert_field(c, r, op, t, sp, R);
    rs = t;
  }
  if (prm.sloppy_codec) {
    HDCG_REQUIRE(scaled, HDCG_ERR_ARG, "sloppy_codec needs a 16-bit sloppy precision (unit-RMS input)");
    codec_roundtrip(c, const_cast<uint4*>(rs), sp, prm.sloppy_codec, R);
  }
  uint4* z = c.scratch(sp, SL_Z, R);
  int nm = 0;
  uint4* t;
  {
    PhaseTimer pt(c, PH_H_SLOPPY);
    cg_shifted(c, sp, rs, z, prm.mirs_shift, prm.mirs_iter, 0.0, prm.mirs_iter, &nm, R);
    t = c.scratch(sp, SL_MP, R);   // the CG's direction is dead now
    apply_mdagm_multi(c, sp, R, z, t, nullptr, -1.0, 1.0, rs);  // t = r - H z
    nm += R;
  }
  if (st) st->n_mdagm_sloppy += nm;
  if (sp == op) {
    apply_Q_multi(c, sp, R, t, y, sp, z, prm, st);
  } else if (scaled && sp == HDCG_F16) {
    // the coarse-grid correction amplifies low modes by up to 1 / lambda_min(H),
    // beyond the FP16 range: y = unscale(z + Q t) is formed in the outer precision
    apply_Q_multi(c, sp, R, t, y, op, z, prm, st, HDCG_F16, dsc(c, D_NREAL), dsc(c, D_TMP));
  } else if (scaled) {
    uint4* zf = c.scratch(HDCG_F32, SL_Z, R);
    uint4* yf = c.scratch(HDCG_F32, SL_MRES, R);
    convert_field(c, z, sp, zf, HDCG_F32, R);
    apply_Q_multi(c, sp, R, t, yf, HDCG_F32, zf, prm, st);
    convert_scaled(c, yf, HDCG_F32, y, op, dsc(c, D_NREAL), dsc(c, D_TMP), 1, R);
  } else {
    uint4* ys = c.scratch(sp, SL_MRES, R);
    apply_Q_multi(c, sp, R, t, ys, sp, z, prm, st);
    convert_field(c, ys, sp, y, op, R);
  }
}

static void start_vector_multi(Ctx& c, int sp, int R, const uint4* b64, uint4* xhi, const hdcg_params& prm,
                               hdcg_stats* st) {
  uint4* bs = c.scratch(sp, SL_RS, R);
  const bool scaled = is_16bit(sp);
  if (scaled) {
    norm2(c, b64, HDCG_F64, 0, dsc(c, D_TMP), R);
    cap_scale(c, b64, HDCG_F64, dsc(c, D_NREAL), dsc(c, D_TMP), SCALED_PEAK,
              reinterpret_cast<unsigned*>(dsc(c, D_AMAX)), R);
    convert_scaled(c, b64, HDCG_F64, bs, sp, dsc(c, D_NREAL), dsc(c, D_TMP), 0, R);
    // x_hi = unscale(Q b_s), prolonged straight into FP64
    apply_Q_multi(c, sp, R, bs, xhi, HDCG_F64, nullptr, prm, st, -1, dsc(c, D_NREAL), dsc(c, D_TMP));
  } else {
    convert_field(c, b64, HDCG_F64, bs, sp, R);
    uint4* x0 = c.scratch(sp, SL_T, R);
    apply_Q_multi(c, sp, R, bs, x0, sp, nullptr, prm, st);
    convert_field(c, x0, sp, xhi, HDCG_F64, R);
  }
}

// r64_k = b_k - H64 x_k for all right-hand sides, one at a time; rr[k] on the
// host; r_k (op) = r64_k
static void true_residual_multi(Ctx& c, int op, int R, const uint4* b64, const uint4* xhi, uint4* r, double* rr,
                                hdcg_stats* st) {
  uint4* r64 = c.scratch(HDCG_F64, SL_R64);
  const size_t f64 = c.field_bytes(HDCG_F64) / 16, fop = c.field_bytes(op) / 16;
  for (int k = 0; k < R; ++k) {
    {
      PhaseTimer pt(c, PH_H_F64);
      residual_df(c, b64 + k * f64, xhi + k * f64, r64);
    }
    norm2(c, r64, HDCG_F64, 0, dsc(c, D_RR) + k);
    if (op != HDCG_F64) convert_field(c, r64, HDCG_F64, r + k * fop, op);
    else copy_field(c, HDCG_F64, r64, r + k * fop);
  }
  if (st) st->n_mdagm_f64 += R;
  HDCG_CUDA(cudaMemcpyAsync(rr, dsc(c, D_RR), R * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
}

static int solve_batch(Ctx& c, const uint4* b64, uint4* x64, int R, double tol, const hdcg_params& prm,
                       hdcg_stats* st) {
  const int op = prm.outer_prec, sp = prm.sloppy_prec;
  const bool adef2 = prm.algorithm == HDCG_ALG_ADEF2;
  HDCG_REQUIRE(R >= 1 && R <= RMAX, HDCG_ERR_ARG, "1..16 right-hand sides per batch");
  HDCG_REQUIRE(op == HDCG_F64 || op == HDCG_F32, HDCG_ERR_ARG, "outer precision must be F64 or F32");
  if (adef2) HDCG_REQUIRE(c.sub && c.coarse, HDCG_ERR_STATE, "A-DEF2 needs a subspace and a coarse operator");
  uint4* xlo = c.scratch(op, SL_XLO, R);
  uint4* r = c.scratch(op, SL_R, R);
  uint4* p = c.scratch(op, SL_P, R);
  uint4* y = c.scratch(op, SL_Y, R);
  uint4* xhi = x64;
  DevMem dmask;
  dmask.ensure(RMAX * sizeof(int));
  int mask[RMAX] = {0};
  auto upload_mask = [&]() {
    HDCG_CUDA(cudaMemcpyAsync(dmask.p, mask, RMAX * sizeof(int), cudaMemcpyHostToDevice, c.stream));
  };
  double bb[RMAX], rr[RMAX], rr_rel[RMAX], stop[RMAX];
  norm2(c, b64, HDCG_F64, 0, dsc(c, D_BB), R);
  HDCG_CUDA(cudaMemcpyAsync(bb, dsc(c, D_BB), R * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
  zero_field(c, xhi, HDCG_F64, R);
  zero_field(c, xlo, op, R);
  if (adef2) start_vector_multi(c, sp, R, b64, xhi, prm, st);
  true_residual_multi(c, op, R, b64, xhi, r, rr, st);
  int nactive = 0;
  for (int k = 0; k < R; ++k) {
    stop[k] = tol * tol * bb[k];
    rr_rel[k] = rr[k];
    mask[k] = (bb[k] > 0.0 && rr[k] > stop[k]) ? 1 : 0;
    nactive += mask[k];
  }
  upload_mask();
  int it = 0;
  int status = nactive ? HDCG_NOT_CONVERGED : HDCG_OK;
  if (nactive) {
    if (adef2) {
      apply_M1_multi(c, op, sp, R, r, y, prm, st);
      copy_fields(c, op, y, p, R);
      redot2(c, op, r, y, nullptr, dsc(c, D_RYN), R);
      HDCG_CUDA(cudaMemcpy2DAsync(dsc(c, D_RY), sizeof(double), dsc(c, D_RYN), 2 * sizeof(double), sizeof(double), R,
                                  cudaMemcpyDeviceToDevice, c.stream));
    } else {
      copy_fields(c, op, r, p, R);
      copy_scalars(c, D_RY, D_RR, R);
    }
  }
  while (nactive && it < prm.maxiter) {
    {
      PhaseTimer pt(c, PH_H_OUTER);
      apply_mdagm_cg(c, op, p, 0.0, xlo, r, dsc(c, D_RY), dsc(c, D_PW), nullptr, dsc(c, D_RR), R,
                     dmask.as<int>());
    }
    st->n_mdagm_outer += R;
    ++it;
    double pw[RMAX];
    HDCG_CUDA(cudaMemcpyAsync(pw, dsc(c, D_PW), R * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    HDCG_CUDA(cudaMemcpyAsync(rr, dsc(c, D_RR), R * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    HDCG_CUDA(cudaStreamSynchronize(c.stream));
    bool need = it >= prm.maxiter;
    for (int k = 0; k < R; ++k) {
      if (!mask[k]) continue;
      HDCG_REQUIRE(std::isfinite(pw[k]) && std::isfinite(rr[k]), HDCG_ERR_NONFINITE, "non-finite residual");
      HDCG_REQUIRE(pw[k] > 0.0, HDCG_ERR_BREAKDOWN, "(p, Hp) <= 0");
      if (rr[k] <= prm.reliable_delta * prm.reliable_delta * rr_rel[k] || rr[k] <= stop[k]) need = true;
    }
    if (need) {
      accum_hi(c, HDCG_F64, xhi, op, xlo, R);
      true_residual_multi(c, op, R, b64, xhi, r, rr, st);
      ++st->reliable_updates;
      nactive = 0;
      for (int k = 0; k < R; ++k) {
        if (!mask[k]) continue;
        rr_rel[k] = rr[k];
        if (rr[k] <= stop[k]) mask[k] = 0;
        nactive += mask[k];
      }
      upload_mask();
      if (!nactive) {
        status = HDCG_OK;
        break;
      }
    }
    if (adef2) {
      // (r, y_old) for the flexible beta, then y_new overwrites y_old
      if (prm.flexible) redot2(c, op, r, y, nullptr, dsc(c, D_RYO), R);
      apply_M1_multi(c, op, sp, R, r, y, prm, st);
      redot2(c, op, r, y, nullptr, dsc(c, D_RYN), R);
      ScalarRef be;
      be.num = dsc(c, D_RYN);
      be.den0 = dsc(c, D_RY);
      be.den1 = prm.flexible ? dsc(c, D_RYO) : nullptr;
      be.stride = 2;
      update_p(c, op, p, y, be, nullptr, R);
      HDCG_CUDA(cudaMemcpy2DAsync(dsc(c, D_RY), sizeof(double), dsc(c, D_RYN), 2 * sizeof(double), sizeof(double), R,
                                  cudaMemcpyDeviceToDevice, c.stream));
    } else {
      ScalarRef be;
      be.num = dsc(c, D_RR);
      be.den0 = dsc(c, D_RY);
      update_p(c, op, p, r, be, nullptr, R);
      copy_scalars(c, D_RY, D_RR, R);
    }
  }
  st->iterations += it;
  double worst = 0.0;
  for (int k = 0; k < R; ++k)
    if (bb[k] > 0.0) worst = std::max(worst, std::sqrt(rr_rel[k] / bb[k]));
  if (worst > st->true_residual) st->true_residual = worst;
  return status;
}

// Device bytes one more right-hand side of a batch needs: FP64 b and x, the
// outer recursion (x_lo, r, p, y and the two intermediate fields of H), the
// preconditioner's fields (r_s, z, the CG's residual and direction, and the
// intermediates of the sloppy H), and host staging of b and x.
static size_t bytes_per_rhs(const Ctx& c, const hdcg_params& prm, bool on_device) {
  const int op = prm.outer_prec, sp = prm.sloppy_prec;
  size_t n = 2 * c.field_bytes(HDCG_F64) + 6 * c.field_bytes(op);
  if (prm.algorithm == HDCG_ALG_ADEF2) n += 4 * c.field_bytes(sp) + (sp != op ? 2 * c.field_bytes(sp) : 0);
  if (!on_device) n += 2 * c.n5 * 12 * sizeof(double2);
  return n;
}

// Right-hand sides per batch: at most 16, and no more than the device memory
// free now (plus what this handle's work fields already hold, which a batch
// reuses) can take, keeping 4 GiB for the library's other buffers.
static int batch_size(Ctx& c, const hdcg_params& prm, int nrhs, bool on_device) {
  if (!prm.batch) return 1;
  size_t freeb = 0, total = 0;
  HDCG_CUDA(cudaMemGetInfo(&freeb, &total));
  // work fields that grow with the batch (and are reused by it when they exist)
  const int op = prm.outer_prec, sp = prm.sloppy_prec;
  size_t held = on_device ? 0 : c.canon_in.bytes + c.canon_out.bytes;
  for (int slot : {(int)SL_B, (int)SL_XHI}) held += c.scratch_f[HDCG_F64][slot].bytes;
  for (int slot : {(int)SL_XLO, (int)SL_R, (int)SL_P, (int)SL_Y, 0, 1}) held += c.scratch_f[op][slot].bytes;
  if (prm.algorithm == HDCG_ALG_ADEF2 && sp != op)
    for (int slot : {(int)SL_RS, (int)SL_Z, (int)SL_MRES, (int)SL_MP, 0, 1}) held += c.scratch_f[sp][slot].bytes;
  // fields that do not grow with the batch but may not exist yet: the
  // double-float residual (five fields), the FP64 residual, the hop autotuner's
  // four temporary fields
  size_t fixed = 0;
  if (!c.scratch_f[HDCG_DF64][5].p) fixed += 5 * c.field_bytes(HDCG_DF64) + c.field_bytes(HDCG_F64);
  fixed += 4 * c.field_bytes(HDCG_DF64);
  const size_t reserve = (size_t(4) << 30) + fixed;
  const size_t avail = freeb + held;
  const size_t per = bytes_per_rhs(c, prm, on_device);
  const size_t fit = avail > reserve ? (avail - reserve) / per : 0;
  return (int)std::max<size_t>(1, std::min<size_t>(std::min<size_t>((size_t)RMAX, (size_t)nrhs), fit));
}

bool is_family_algorithm(int alg);
int solve_family(Ctx& c, const uint4* b64, uint4* x64, double tol, const hdcg_params& prm, hdcg_stats* st);

int solve(Ctx& c, const void* b, void* x, int nrhs, double tol, const hdcg_params& prm, hdcg_stats* st,
          bool on_device) {
  HDCG_REQUIRE(nrhs >= 1, HDCG_ERR_ARG, "nrhs >= 1");
  HDCG_REQUIRE(tol > 0.0, HDCG_ERR_ARG, "tol > 0");
  HDCG_REQUIRE(c.have_gauge && c.have_dwf, HDCG_ERR_STATE, "gauge field and DWF parameters required");
  const auto t0 = std::chrono::steady_clock::now();
  std::memset(st, 0, sizeof(*st));
  const size_t canon = c.n5 * 12 * sizeof(double2);
  int worst = HDCG_OK;
  {
    const double nreal = (double)c.n5 * 24.0;
    HDCG_CUDA(cudaMemcpyAsync(dsc(c, D_NREAL), &nreal, sizeof(double), cudaMemcpyHostToDevice, c.stream));
  }
  const bool family = is_family_algorithm(prm.algorithm);
  const int chunk = family ? 1 : batch_size(c, prm, nrhs, on_device);
  st->batch_rhs = chunk;
  for (int k0 = 0; k0 < nrhs; k0 += chunk) {
    const int R = std::min(chunk, nrhs - k0);
    const char* bk = reinterpret_cast<const char*>(b) + k0 * canon;
    char* xk = reinterpret_cast<char*>(x) + k0 * canon;
    uint4* b64 = c.scratch(HDCG_F64, SL_B, R);
    uint4* x64 = c.scratch(HDCG_F64, SL_XHI, R);
    if (on_device) {
      canon_to_internal(c, bk, HDCG_F64, b64, HDCG_F64, R);
    } else {
      c.canon_in.ensure(canon * R);
      HDCG_CUDA(cudaMemcpyAsync(c.canon_in.p, bk, canon * R, cudaMemcpyHostToDevice, c.stream));
      canon_to_internal(c, c.canon_in.p, HDCG_F64, b64, HDCG_F64, R);
    }
    int rc;
    {
      PhaseTimer pt(c, PH_TOTAL);
      rc = family ? solve_family(c, b64, x64, tol, prm, st)
           : R == 1 ? solve_one(c, b64, x64, tol, prm, st) : solve_batch(c, b64, x64, R, tol, prm, st);
    }
    if (rc != HDCG_OK) worst = rc;
    if (on_device) {
      internal_to_canon(c, x64, HDCG_F64, xk, HDCG_F64, R);
    } else {
      c.canon_out.ensure(canon * R);
      internal_to_canon(c, x64, HDCG_F64, c.canon_out.p, HDCG_F64, R);
      HDCG_CUDA(cudaMemcpyAsync(xk, c.canon_out.p, canon * R, cudaMemcpyDeviceToHost, c.stream));
    }
  }
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
  st->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  st->status = worst;
  return worst;
}

// ---------------------------------------------------------------------------
// subspace by inverse iteration and the coarse operator
// ---------------------------------------------------------------------------
// v <- (H + shift)^-1 v by CG in precision wp (v stored in vprec)
void inverse_step(Ctx& c, int wp, uint4* v, int vprec, double shift, double tol, int maxiter) {
  uint4* bk = c.scratch(wp, SL_CGB);
  uint4* xk = c.scratch(wp, SL_CGX);
  convert_field(c, v, vprec, bk, wp);
  cg_shifted(c, wp, bk, xk, shift, 0, tol, maxiter, nullptr);
  convert_field(c, xk, wp, v, vprec);
}

void build_subspace(Ctx& c, const hdcg_subspace_params& p) {
  HDCG_REQUIRE(c.have_gauge && c.have_dwf, HDCG_ERR_STATE, "gauge field and DWF parameters required");
  for (int mu = 0; mu < 4; ++mu)
    HDCG_REQUIRE(p.block[mu] >= 4, HDCG_ERR_ARG, "block extents must be >= 4 (Sec. 5.1)");
  if (!c.sub) c.sub = new Subspace();
  Subspace& s = *c.sub;
  // a 16-bit subspace is built in FP32 and rounded once at the end: inverse
  // iteration makes the block pieces nearly dependent, which 16-bit storage
  // would blur before the block orthonormalisation can separate them
  const bool round_at_end = p.prec == HDCG_F16;
  subspace_init(c, s, p.block, p.nvec, round_at_end ? HDCG_F32 : p.prec);
  subspace_noise(c, s, p.seed);
  const int wp = p.prec == HDCG_F64 ? HDCG_F64 : HDCG_F32;
  for (int step = 0; step < p.inv_steps; ++step) {
    for (int k = 0; k < s.nvec; ++k) inverse_step(c, wp, s.vec(c, k), s.prec, p.inv_shift, p.inv_tol, p.inv_maxiter);
    block_orthonormalise(c, s);
  }
  if (p.inv_steps <= 0) block_orthonormalise(c, s);
  if (round_at_end) {
    DevMem v32;
    std::swap(v32.p, s.vecs.p);
    std::swap(v32.bytes, s.vecs.bytes);
    s.prec = HDCG_F16;
    s.vecs.ensure((size_t)s.nvec * s.vec_bytes(c));
    convert_field(c, v32.as<uint4>(), HDCG_F32, s.vecs.as<uint4>(), HDCG_F16, s.nvec);
    block_orthonormalise(c, s);
  }
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
}

void build_coarse(Ctx& c, int prec) {
  HDCG_REQUIRE(c.sub, HDCG_ERR_STATE, "no subspace");
  HDCG_REQUIRE((prec == HDCG_F64) == (c.sub->prec == HDCG_F64), HDCG_ERR_ARG,
               "the coarse operator is FP64 exactly when the subspace is FP64");
  if (!c.coarse) c.coarse = new Coarse();
  coarse_init(c, *c.coarse, *c.sub, prec);
  coarse_assemble(c, *c.coarse, *c.sub, prec == HDCG_F64 ? HDCG_F64 : HDCG_F32);
}

void set_coarse(Ctx& c, const void* A, int prec, int on_device) {
  HDCG_REQUIRE(c.sub, HDCG_ERR_STATE, "no subspace (it fixes the blocking and Nvec)");
  HDCG_REQUIRE((prec == HDCG_F64) == (c.sub->prec == HDCG_F64), HDCG_ERR_ARG,
               "the coarse operator is FP64 exactly when the subspace is FP64");
  if (!c.coarse) c.coarse = new Coarse();
  coarse_init(c, *c.coarse, *c.sub, prec);
  coarse_import(c, *c.coarse, A, on_device);
}

}  // namespace hdcg
