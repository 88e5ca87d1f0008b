/*
 * hdcg.h -- C ABI of the GB300 (sm_103a) hierarchically deflated CG library.
 *
 * The calls follow the statement of the problem in Boyle, "Hierarchically
 * deflated conjugate gradient" (arXiv 1402.2585): a 4D lattice with a fifth
 * dimension of extent Ls, an SU(3) gauge field, the domain-wall / Moebius
 * parameters (M5, b, c, m), the red-black preconditioned Hermitian operator
 * H = Mpc^dag Mpc (Sec. 4), a blocked deflation subspace (Sec. 2), the little
 * Dirac operator A (Sec. 2, Sec. 5.1, Sec. 5.1.1) and the A-DEF2 solve
 * (Fig. pcg_general, Table algos).
 *
 * Conventions shared by every call
 * --------------------------------
 * Return value: HDCG_OK (0) on success; HDCG_NOT_CONVERGED (+1) when a solve
 *   stops at its iteration limit (x then holds the last iterate); a negative
 *   HDCG_ERR_* code otherwise.  hdcg_last_error() gives a one-line reason.
 *   A call that fails leaves the handle usable unless it reports
 *   HDCG_ERR_CUDA (a CUDA error may poison the context).
 * Lattice: extents (Lx, Ly, Lz, Lt) all even; site lex = x + Lx(y + Ly(z + Lz t));
 *   parity (x+y+z+t) mod 2; checkerboard index cb = lex >> 1.  The solved system
 *   lives on the odd checkerboard.  Ls must be a power of two between 2 and 32.
 * Canonical fermion field ("odd field"): [cb][s][spin 4][colour 3] complex,
 *   real and imaginary parts interleaved, element type given by a precision
 *   code (HDCG_F64: double, HDCG_F32: float, HDCG_F16: IEEE half,
 *   HDCG_BF16 / HDCG_BF16T: bfloat16).  Size (V/2) * Ls * 12 complex.
 *   Gamma matrices: chiral basis, gamma5 = diag(1, 1, -1, -1).
 * Canonical gauge field: [lex][mu = x, y, z, t][row 3][col 3] complex double;
 *   U_mu(x) links x to x + mu.
 * Canonical coarse vector: [coarse site][Nvec] complex; coarse sites are the
 *   blocks in lexicographic order of their block coordinates.
 * Canonical coarse operator: [coarse site a][l][j][k] complex double with
 *   A[a][l][j][k] = <phi_j^a | H | phi_k^{a + delta_l}>,
 *   l = (dx+1) + 3 (dy+1) + 9 (dz+1) + 27 (dt+1), delta in {-1, 0, 1}^4.
 *   Along a coarse extent of 2 only delta in {0, +1} is stored (delta = -1
 *   aliases +1), along an extent of 1 only delta = 0; other entries are zero.
 * Pointers: device pointers on the handle's stream unless a call takes an
 *   on_device flag (0 = host memory).  The caller owns every buffer it passes;
 *   the handle owns the internal copies and work space it allocates.
 *   Calls are asynchronous on the stream only where stated; the others
 *   synchronise the stream before returning.
 */
#ifndef HDCG_H
#define HDCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* precision codes: storage type; arithmetic is FP32 for 16/32-bit storage, FP64 for FP64 */
#define HDCG_F64   0
#define HDCG_F32   1
#define HDCG_F16   2   /* IEEE half, round to nearest even */
#define HDCG_BF16  3   /* bfloat16 (8-bit exponent, 7-bit mantissa), round to nearest even */
#define HDCG_BF16T 4   /* bfloat16 by truncating the float32 word to its top 16 bits (Sec. 6.5) */
#define HDCG_DF64  5   /* hdcg_apply_mpc / hdcg_apply_mdagm only: complex double buffers, operator
                          stored and computed as double-float (hi + lo float32 pairs, about 48
                          significant bits) on the FP32 units; the FP64-accurate operator the
                          solver uses for its true residuals */

/* return codes */
#define HDCG_OK             0
#define HDCG_NOT_CONVERGED  1
#define HDCG_ERR_ARG       -1  /* invalid argument or unsupported size */
#define HDCG_ERR_OOM       -2  /* device allocation failed */
#define HDCG_ERR_CUDA      -3  /* a CUDA call failed */
#define HDCG_ERR_NONFINITE -4  /* a residual or inner product became NaN/Inf */
#define HDCG_ERR_BREAKDOWN -5  /* (p, Hp) <= 0 or (r, y) <= 0 in a Krylov step */
#define HDCG_ERR_TIMEOUT   -6  /* a bounded device-side wait expired (tensor-core pipeline); the
                                 context stays usable, the result of that call is undefined */
#define HDCG_ERR_STATE     -7  /* prerequisite missing (no gauge field, no subspace, ...) */

/* solver algorithms */
#define HDCG_ALG_CG    0  /* plain CG on H (the red-black normal-equation baseline) */
#define HDCG_ALG_ADEF2 1  /* A-DEF2: V_start = Qb + P_R x, M1 = P_R M_IRS + Q (Table algos) */
/* The rest of Table algos (Sec. 4.5, Fig. pcg_general), with Q = P A^-1 R,
 * P_L = 1 - H Q, P_R = 1 - Q H and the smoother M of hdcg_params.smoother.
 * These run the generalised PCG one right-hand side at a time with every
 * field and operator in outer_prec (F64 or F32; sloppy_prec, batch and
 * reliable_delta are not used), stop on the recursive residual, and report
 * the FP64 true residual. */
#define HDCG_ALG_PREC   2   /* M1 = M */
#define HDCG_ALG_AD     3   /* M1 = M + Q */
#define HDCG_ALG_DEF1   4   /* M1 = M, M3 = P_L (start residual projected), V_end = Q b + P_R x */
#define HDCG_ALG_DEF2   5   /* M1 = M, M2 = P_R, V_start = Q b + P_R x */
#define HDCG_ALG_ADEF1  6   /* M1 = M P_L + Q (M2 = 1) */
#define HDCG_ALG_BNN    7   /* M1 = P_R M P_L + Q */
#define HDCG_ALG_BNN_DEF2START 8   /* BNN from V_start = Q b + P_R x */
#define HDCG_ALG_V11    9   /* M1 = M P_L + P_R M + Q - M P_L H M (symmetric two-grid cycle) */
#define HDCG_ALG_MSSDEF 10  /* A-DEF2 with M = 1 (the little Dirac operator alone) */
#define HDCG_ALG_ADEF2_FAMILY 11  /* A-DEF2 in the generalised PCG (same algorithm as
                                     HDCG_ALG_ADEF2 without its mixed precision) */

/* smoothers of the family solves (Table preconditioner) */
#define HDCG_SMOOTHER_MIRS      0  /* mirs_iter CG iterations on H + mirs_shift from zero */
#define HDCG_SMOOTHER_MIRSPOLY  1  /* the same CG's alpha_k, beta_k frozen from one pass on
                                      the right-hand side b and replayed: a fixed polynomial
                                      in H, linear and Hermitian */
#define HDCG_SMOOTHER_CHEBYSHEV 2  /* p(H), 1 - x p(x) = T_n((theta - x)/delta) / T_n(theta/delta)
                                      on [cheb_lo, cheb_hi], n = cheb_order */
#define HDCG_SMOOTHER_NONE      3  /* M = 1 */

typedef struct hdcg_ctx* hdcg_t;

/* Create a lattice of extents dims[4] with fifth-dimension extent Ls.
 * antiperiodic_t: 1 multiplies hops across the time boundary by -1.
 * cuda_stream: cudaStream_t to run on (NULL = legacy default stream).
 * Allocates only small index tables.  Errors: HDCG_ERR_ARG (odd or < 2 extent,
 * Ls not a power of two in [2, 32]), HDCG_ERR_OOM, HDCG_ERR_CUDA. */
int hdcg_create(hdcg_t* h, const int dims[4], int Ls, int antiperiodic_t, void* cuda_stream);

/* Domain-wall / Moebius parameters (Sec. 4 operator; Shamir: b = 1, c = 0).
 * D psi_s = D_W (K psi)_s + ((1 - P_s) psi)_s, K = b + c P_s,
 * (P_s psi)_s = P_- psi_{s+1} + P_+ psi_{s-1}, psi_{Ls} -> -m psi_0, psi_{-1} -> -m psi_{Ls-1},
 * D_W = (4 - M5) - Dh/2.  Errors: HDCG_ERR_ARG if M_ee is singular. */
int hdcg_set_dwf(hdcg_t h, double M5, double b, double c, double mass);

/* Upload the gauge field (canonical, complex double, host or device).  The
 * library keeps its own copies in FP64, FP32 and 16-bit link layouts.  The
 * links are reused across all Ls slices (Sec. 6.5).  Synchronous. */
int hdcg_set_gauge(hdcg_t h, const void* U, int on_device);

/* out = Mpc in (dagger = 0) or Mpc^dag in (dagger = 1) on odd fields, where
 * Mpc = M_oo - M_oe M_ee^-1 M_eo (Sec. 4).  in/out: canonical odd fields of
 * precision prec on the device, distinct buffers.  Asynchronous on the stream. */
int hdcg_apply_mpc(hdcg_t h, const void* in, void* out, int dagger, int prec);

/* The full domain wall system D psi = eta on both checkerboards and its
 * Schur-form reduction (Sec. 4): D = [[M_ee, M_eo], [M_oe, M_oo]] on (even, odd)
 * sites, M_ee = M_oo = (4 - M5) K + 1 - P_s, M_eo = M_oe = -Dh K / 2.  The odd
 * half of psi solves H psi_o = b with
 *   b = Mpc^dag (eta_o - M_oe M_ee^-1 eta_e)          (hdcg_prep_source),
 * and the even half is
 *   psi_e = M_ee^-1 (eta_e - M_eo psi_o)              (hdcg_reconstruct).
 * Every field is canonical complex double [cb][s][spin][colour] (the even
 * field indexed by the even checkerboard, cb = lex >> 1 of its even sites),
 * host or device (on_device), caller-owned.  FP64 arithmetic.  Synchronous. */
int hdcg_prep_source(hdcg_t h, const void* eta_e, const void* eta_o, void* b, int on_device);
int hdcg_reconstruct(hdcg_t h, const void* eta_e, const void* psi_o, void* psi_e, int on_device);

/* out = H in = Mpc^dag Mpc in (Sec. 4).  If pHp is not NULL it receives
 * (in, H in) = |Mpc in|^2 accumulated in FP64 (then the call synchronises). */
int hdcg_apply_mdagm(hdcg_t h, const void* in, void* out, int prec, double* pHp);

/* ---------------------------------------------------------------------------
 * Deflation subspace and little Dirac operator (Sec. 2, Sec. 5.1)
 * ------------------------------------------------------------------------- */
typedef struct {
    int block[4];        /* block extents; each >= 4 and dividing the lattice extent */
    int nvec;            /* number of subspace vectors, 1..64 */
    int prec;            /* storage precision of the subspace: HDCG_F64, _F32 or _F16 */
    int inv_steps;       /* inverse-iteration steps (each followed by block Gram-Schmidt) */
    double inv_shift;    /* lambda_s: each step applies (H + lambda_s)^-1 */
    double inv_tol;      /* relative residual of the CG in each step */
    int inv_maxiter;     /* iteration cap of that CG */
    uint64_t seed;       /* Gaussian start vectors: splitmix64 counter stream + Box-Muller */
    int level;           /* 1 (or 0): blocks of the fine lattice, vectors of H;
                            2: blocks of the coarse lattice, vectors of the little Dirac
                            operator A (block extents >= 1 dividing the coarse extents,
                            nvec <= 64, prec HDCG_F32); see hdcg_build_coarse */
    int method;          /* level 1: HDCG_SUBSPACE_INVITER (0) as above, or
                            HDCG_SUBSPACE_RATIONAL (1): the rational low-pass filter of
                            Sec. 4.2 (Eq. ratfilt); HDCG_SUBSPACE_CONTINUE (2): inverse
                            iteration started from the current subspace instead of noise
                            (the second pass of the two-stage generation, Sec. 4.2) */
    double filter_lambda;/* RATIONAL: phi = prod_{i < filter_order} (H + lambda + i eps)^-1 eta */
    double filter_eps;   /*   eps > 0 (any value for order 1) */
    int filter_order;    /*   1..8 (the paper: 4) */
    int surface_depth;   /* RATIONAL and CONTINUE: > 0 keeps only the s-slices
                            s < depth and s >= Ls - depth (SubspaceSurfaceDepth,
                            Table FineSubspaceParams); 0 keeps all */
} hdcg_subspace_params;

#define HDCG_SUBSPACE_INVITER 0
#define HDCG_SUBSPACE_RATIONAL 1
#define HDCG_SUBSPACE_CONTINUE 2

/* Build the subspace by inverse iteration from Gaussian noise, with block
 * Gram-Schmidt (FP64 arithmetic) after each step (Sec. 2; inverse iteration
 * as named in Sec. 1 and Sec. 5.2.1).  Level 1: vectors of H on the fine
 * lattice, each step a CG on H + inv_shift.
 * Level 1, method HDCG_SUBSPACE_RATIONAL (Sec. 4.2): vector k starts from 4D
 * Gaussian noise xi_k (the splitmix64 stream seed, canonical order
 * [k][cb][spin][colour]) placed as P_- xi at s = 0 and P_+ xi at s = Ls - 1,
 * and is filtered by prod_i (H + lambda + i eps)^-1 = sum_i c_i (H + lambda +
 * i eps)^-1, c_i = prod_{j != i} 1 / (sigma_j - sigma_i), all shifts from one
 * multi-shift CG to relative residual inv_tol (cap inv_maxiter), then
 * truncated to surface_depth and block-orthonormalised.  Method
 * HDCG_SUBSPACE_CONTINUE applies inv_steps inverse-iteration steps of shift
 * inv_shift to the current subspace (e.g. one promoted by
 * hdcg_promote_subspace), then the truncation and block Gram-Schmidt.
 * Level 2 (three-level HDCG): the same construction on the coarse lattice, Sec. 2 applied to the little Dirac
 * operator; each step solves (A + inv_shift) for up to 16 vectors at once
 * (coarse CG), and the start vectors are the splitmix64 stream seed in
 * canonical order [k][Vc][Nvec].  Level 2 needs the level-1 operator (FP32 or
 * FP16).  Synchronous. */
int hdcg_build_subspace(hdcg_t h, const hdcg_subspace_params* p);

/* The first pass of the two-stage generation (Sec. 4.2): the level-1 subspace
 * of src, a handle on the same 4D lattice with fifth extent Ls1 <= Ls (its own
 * mass; e.g. built with HDCG_SUBSPACE_RATIONAL), promoted into h: the slices
 * s < ceil(Ls1 / 2) stay at s, the others move to s + Ls - Ls1 (each keeps its
 * distance to its wall), the bulk between is zero; stored in prec (F64, F32 or
 * F16) with src's blocking and block-orthonormalised.  Both handles on the
 * current device; src is not modified.  The second pass is
 * hdcg_build_subspace with HDCG_SUBSPACE_CONTINUE.  Synchronous. */
int hdcg_promote_subspace(hdcg_t h, hdcg_t src, int prec);

/* Upload a subspace: level 1: phi canonical complex double [nvec][odd field];
 * level 2: phi canonical complex double [nvec][Vc][Nvec] (stored FP32; prec must
 * be HDCG_F32) with level-2 blocks block[4] of the coarse lattice.  Host or
 * device.  It is block-orthonormalised again (FP64) before use unless
 * already_orthonormal is 1.  Synchronous. */
int hdcg_set_subspace(hdcg_t h, int level, const int block[4], int nvec, int prec, const void* phi,
                      int on_device, int already_orthonormal);

/* Copy the subspace of a level out (canonical complex double, host).  Synchronous. */
int hdcg_get_subspace(hdcg_t h, int level, void* phi_host);

/* Level 1: assemble A = R H P by the Fourier trick of Sec. 5.1.1 (81 phased H
 * applies per subspace vector, inverted one dimension at a time); prec is the
 * storage precision of A (HDCG_F64, _F32 or _F16; an FP16 A keeps an FP32 copy
 * for level 2).  Rebuilding A keeps a level-2 subspace of the same geometry and
 * drops the level-2 operator.
 * Level 2 (three-level HDCG): A2 = P2^dag A P2 on the level-2 lattice, the
 * Galerkin product of Sec. 2 one level down, contracted directly from the
 * blocks of A in FP64 (an 81-point stencil again, same canonical layout and
 * aliasing rule as A), and its dense inverse by Gauss-Jordan elimination,
 * stored in prec (HDCG_F32 or HDCG_F64; Vc2 * Nvec2 <= 65536).  From then on
 * every coarse solve (the inversion of A inside Q, and hdcg_coarse_solve) is
 * A-DEF2 on A with Q2 = P2 A2^-1 R2 and M = 1 (Fig. pcg_general, Table algos):
 * x0 = Q2 b, y = r + Q2 (r - A r), flexible beta; or with M the Chebyshev
 * polynomial of Q_trunc (hdcg_set_coarse_preconditioner): y = z + Q2 (r - A z),
 * z = M r.  HDCG_ERR_BREAKDOWN if A2 has
 * a non-positive diagonal or a zero pivot.  Synchronous. */
int hdcg_build_coarse(hdcg_t h, int level, int prec);

/* Canonical layout of A: complex double [Vc][81][j][k], block (a, l) couples
 * coarse site a to its neighbour a + delta_l with
 * l = (dx+1) + 3 (dy+1) + 9 (dz+1) + 27 (dt+1), delta in {-1,0,1}^4, coarse
 * sites lexicographic in the block coordinates (x fastest); y_a = sum_l
 * A[a][l] x_{a+delta_l}.  Along a coarse extent of 2 only the offsets 0, +1
 * are stored (-1 is the same neighbour), along an extent of 1 only 0; the
 * other blocks are zero.  */

/* Copy A (level 1) or A2 (level 2) out in the canonical layout (complex double,
 * host: [Vc][81][Nvec][Nvec] or [Vc2][81][Nvec2][Nvec2]).  Synchronous. */
int hdcg_get_coarse(hdcg_t h, int level, void* A_host);

/* Level-2 restriction c2 = R2 x (c2[b][k] = <phi2_k^b, x>) and prolongation
 * x = P2 c2 for nrhs (1..16) vectors: x canonical [nrhs][Vc][Nvec], c2
 * [nrhs][Vc2][Nvec2], complex double, device (FP32 arithmetic).  Synchronous. */
int hdcg_restrict_coarse(hdcg_t h, const void* x, void* c2, int nrhs);
int hdcg_prolong_coarse(hdcg_t h, const void* c2, void* x, int nrhs);

/* Upload a little Dirac operator in the canonical layout (host or device
 * pointer, complex double), stored in precision prec (F64, F32 or F16; round
 * to nearest).  A subspace must be set first: it fixes the blocking, Vc and
 * Nvec; prec is F64 exactly when the subspace is.  Replaces any operator
 * built before.  Synchronous. */
int hdcg_set_coarse(hdcg_t h, const void* A, int prec, int on_device);

/* c = R v (c[b][k] = <phi_k^b, v>), v a canonical odd field of precision prec on
 * the device, c a canonical coarse vector (complex double, device). */
int hdcg_restrict(hdcg_t h, const void* v, int prec, void* c);
/* v = P c = sum_k c[b(x)][k] phi_k(x); c complex double (device), v precision prec. */
int hdcg_prolong(hdcg_t h, const void* c, void* v, int prec);
/* y = A x on canonical coarse vectors (complex double, device). */
int hdcg_coarse_apply(hdcg_t h, const void* x, void* y);

/* Y = A X for nrhs (1..16) coarse vectors at once (Sec. 5.1 stencil, one read of
 * A for all of them).  x, y: canonical [nrhs][Vc][Nvec] complex double, device.
 * FP16 and FP32 operators (Nvec <= 64) run on the tensor cores (tcgen05,
 * FP32 accumulation; an FP32 A as an FP16 hi + lo pair, two MMAs per tile; X
 * enters as a scaled FP16 hi + lo pair per value, about 22 significant bits),
 * FP64 operators on the CUDA cores.  HDCG_ERR_TIMEOUT if a device-side
 * pipeline wait expired.  Synchronous. */
int hdcg_coarse_apply_multi(hdcg_t h, const void* x, void* y, int nrhs);

/* Solve A x = b on the coarse level for nrhs (1..16) right-hand sides to the
 * relative residual tol (at most maxiter iterations): A-DEF2 with the level-2
 * operator when one was built (hdcg_build_coarse level 2), else A-DEF1 with
 * the second-level deflation space when one was built, otherwise CG (the inner
 * inversion of Q, Sec. 2).  b, x: canonical [nrhs][Vc][Nvec] complex double,
 * device; x is overwritten (zero start).  *iterations (nullable) receives the
 * lockstep iteration count.  HDCG_ERR_BREAKDOWN if the level-2 A-DEF2 solve
 * met (p, A p) <= 0 or a non-finite residual before the tolerance (inside
 * hdcg_solve the preconditioner keeps that right-hand side's last iterate
 * instead).  Synchronous. */
int hdcg_coarse_solve(hdcg_t h, const void* b, void* x, int nrhs, double tol, int maxiter, int* iterations);

/* y = A x exactly like hdcg_coarse_apply, but without allocating any device
 * memory: for callers that cannot call cudaMalloc on this path (for example a
 * host code that hands all device memory to its own pool allocator, or one
 * that must not grow its footprint while other work is resident).  The paper
 * has no counterpart; it is a property of this library's interface.
 * Scratch (the coarse vectors in the working precision and three partial
 * products) lives in a fixed 32 MiB device array compiled into the library,
 * which every GPU that loads the library holds until the process exits.
 * Limit: 838,860 coarse unknowns (Vc * Nvec) with an FP32/FP16 coarse
 * operator, 699,050 with FP64; larger operators are rejected with
 * HDCG_ERR_ARG and a message giving the bytes needed.  A handle's first call
 * looks up the array's device address with the current device (again if the
 * current device has changed since); make that first call before any stream
 * capture.  All calls on a device share the array and it keeps the last
 * call's contents: calls that overlap on the GPU (several streams or host
 * threads) race.  x, y: canonical coarse vectors, complex double, device.
 * Synchronous: the call waits for its stream before returning. */
int hdcg_coarse_apply_noalloc(hdcg_t h, const void* x, void* y);

/* High-mode preconditioner of the little Dirac operator (Sec. 5.2, "Truncated
 * little Dirac operator as preconditioner"; Table hierarchy: order 16 on
 * [0.5, 45]): M = p(Q_trunc + shift), Q_trunc the blocks of A within one block
 * hop (self and the eight nearest neighbours; on an extent of 2 the stored
 * offsets only), p the Chebyshev-acceleration polynomial of degree order - 1
 * on [lo, hi], 1 - x p(x) = T_order((theta - x)/delta) / T_order(theta/delta).
 * hi <= 0 takes 1.1 times a power-iteration estimate of the largest eigenvalue
 * of Q_trunc + shift (M is positive definite while that bound holds); lo <= 0
 * takes hi |lo| (lo < 0) or hi / 90 (lo = 0, the paper's ratio).  interval
 * (nullable, 2 doubles) receives [lo, hi].  From then on the level-1 solve
 * with a level-2 operator smooths with M: y = z + Q2 (r - A z), z = M r.
 * order 0 removes it; rebuilding A removes it too.  Needs an FP32 or FP16 A.
 * Synchronous. */
int hdcg_set_coarse_preconditioner(hdcg_t h, int order, double lo, double hi, double shift, double* interval);

/* y = M x with the preconditioner above, nrhs (1..16) canonical coarse vectors
 * [nrhs][Vc][Nvec] complex double on the device (FP32 arithmetic).  Synchronous. */
int hdcg_coarse_precondition(hdcg_t h, const void* x, void* y, int nrhs);

/* Second-level (global) deflation of the little Dirac operator (Sec. 5.2,
 * "Little Dirac operator deflation"): nvec Gaussian start vectors (splitmix64
 * stream seed, canonical order [k][Vc][Nvec], as for the subspace) refined by
 * inv_steps steps of (A + shift)^-1 (coarse CG to relative residual tol, at
 * most maxiter iterations), each followed by a global orthonormalisation
 * (Cholesky QR, twice, FP64 Gram), then prediagonalised by Rayleigh-Ritz
 * (dense Hermitian eigensolver on the host) so that Z^dag A Z = diag(lam).
 * The paper uses about 128-160 vectors (Table optimised: LdopDeflVecs 160,
 * LittleDopSolverResidualSubspace 1e-7, three shifted inverse-iteration steps).
 * Afterwards every coarse solve is A-DEF1 with these vectors (M_1 = P_L + Q,
 * M_2 = M_3 = 1, using the stored A Z).  nvec = 0 removes the space.  Needs an
 * FP32 or FP16 little Dirac operator (vectors are FP32).  Synchronous. */
typedef struct {
    int nvec;          /* number of global deflation vectors (<= 256) */
    int inv_steps;     /* inverse-iteration steps */
    double shift;      /* shift of (A + shift)^-1; a negative value means |shift| times the
                          mean diagonal element of A */
    double tol;        /* coarse CG relative residual of each step */
    int maxiter;       /* coarse CG iteration cap of each step */
    uint64_t seed;     /* start vectors */
} hdcg_ldop_params;

int hdcg_build_coarse_deflation(hdcg_t h, const hdcg_ldop_params* p);

/* The Ritz values lam (nvec doubles, ascending; host) and optionally the
 * vectors Z (canonical complex double [nvec][Vc][Nvec], host; may be NULL).
 * Pairs with lam <= 1e-7 lam_max (the computed operator need not be positive
 * definite at the bottom of its spectrum at light masses) are left out of the
 * deflation and reported as lam = +inf. */
int hdcg_get_coarse_deflation(hdcg_t h, double* lam_host, void* Z_host);

/* The dense third level's diagonalisation (the "prediagonalised" global level
 * of Sec. 5.2): eigenvalues w (ascending) and eigenvectors V (columns,
 * complex double row-major n x n, may be NULL) of the Hermitian part of H
 * (complex double row-major n x n), by cyclic complex Jacobi rotations on the
 * host.  No handle and no device work.  HDCG_ERR_ARG for n outside 1..4096
 * or NULL H / w. */
int hdcg_dense_heev(int n, const double* H, double* w, double* V);

/* ---------------------------------------------------------------------------
 * Solve H x = b
 * ------------------------------------------------------------------------- */
typedef struct {
    int algorithm;         /* HDCG_ALG_CG or HDCG_ALG_ADEF2 */
    int outer_prec;        /* operator precision of the outer iteration (F64 or F32) */
    int sloppy_prec;       /* precision of M_IRS and of the operator inside M1 */
    int mirs_iter;         /* M_IRS CG iterations (Table optimised: 7) */
    double mirs_shift;     /* M_IRS infra-red shift lambda (Table optimised: 1.0) */
    double coarse_tol;     /* relative residual of the coarse CG (Table optimised: 0.04) */
    int coarse_maxiter;
    int flexible;          /* 1: flexible (Polak-Ribiere) beta; 0: standard PCG beta */
    int maxiter;           /* outer iteration cap */
    double reliable_delta; /* FP64 true-residual update when |r| falls by this factor */
    int batch;             /* nrhs > 1: 1 solves up to 16 right-hand sides in lockstep (one
                              launch per step covers all of them, the coarse level reads the
                              subspace and A once for all), as many per batch as the free
                              device memory takes (hdcg_stats.batch_rhs); 0 solves them one
                              after another */
    int sloppy_codec;      /* the preconditioner's input (unit-RMS, 16-bit sloppy precision)
                              passes through a reduced-precision codec of Sec. 6.5 before M_IRS,
                              the precision of the paper's compressed preconditioner
                              communication: 0 none, 1 each FP32 word truncated to 16 bits,
                              2 8-bit integers with an FP16 prefactor per 5D site */
    int smoother;          /* family solves (algorithm >= 2): HDCG_SMOOTHER_* */
    int cheb_order;        /* HDCG_SMOOTHER_CHEBYSHEV: order n (>= 1) and interval */
    double cheb_lo, cheb_hi;
} hdcg_params;

typedef struct {
    int iterations;            /* outer iterations */
    int coarse_iterations;     /* total coarse CG iterations */
    int coarse_iterations_max; /* largest single coarse solve */
    int n_mdagm_outer;         /* H applies in the outer precision */
    int n_mdagm_sloppy;        /* H applies inside the preconditioner */
    int n_mdagm_f64;           /* FP64 true-residual H applies */
    int reliable_updates;
    int status;                /* return code of the solve */
    double true_residual;      /* |b - H x| / |b| in FP64 at exit (max over rhs) */
    double seconds;            /* wall time of the solve */
    int batch_rhs;             /* right-hand sides solved together per batch (memory permitting) */
} hdcg_stats;

/* Fill p with the defaults (A-DEF2, FP32 outer, FP32 sloppy, M_IRS(7, 1.0),
 * coarse tol 0.04, flexible, reliable delta 0.01, batched). */
void hdcg_default_params(hdcg_params* p);

/* Solve H x = b for nrhs right-hand sides to |b - H x| / |b| <= tol (true FP64
 * residual).  b, x: nrhs consecutive canonical odd fields, complex double, on
 * the device (on_device = 1) or host (0).  x is overwritten (zero start).
 * HDCG_ALG_ADEF2 needs a subspace and a coarse operator.  Synchronous. */
int hdcg_solve(hdcg_t h, const void* b, void* x, int nrhs, double tol, const hdcg_params* p,
               hdcg_stats* st, int on_device);

/* The 8-bit spinor codec of Sec. 6.5 (Table sloppy's proposal): every 5D site
 * of nfields canonical odd fields (complex double, device) becomes an FP16
 * prefactor p = fp16(max |real| of the site) (round to nearest even) and 24
 * signed bytes q = clip(rint(127 v / p), -127, 127); decoding gives q p / 127.
 * scale: [nfields][cb][s] IEEE half; q: [nfields][cb][s][24] int8 (the 24
 * reals in canonical order).  FP64 arithmetic.  Asynchronous on the stream.
 * Range: a site whose largest |real| rounds beyond FP16's 65504 gets an
 * infinite prefactor and decodes to NaN (the solver's codec input is scaled to
 * unit RMS first, far inside the range). */
int hdcg_encode_i8(hdcg_t h, const void* in, void* scale, void* q, int nfields);
int hdcg_decode_i8(hdcg_t h, const void* scale, const void* q, void* out, int nfields);

/* ---------------------------------------------------------------------------
 * Instrumentation
 * ------------------------------------------------------------------------- */
/* Enable (1) / disable (0) CUDA-event timing of every fine-operator hop launch. */
int hdcg_set_profiling(hdcg_t h, int on);
/* Launch count, summed device time (ms) and algorithmic bytes of the fine
 * hop kernels recorded since profiling was enabled, per storage precision
 * (prec).  bytes counts everything the launches must move, fused epilogues
 * included (CG update, shifted term); op_bytes (nullable) only the operator's
 * own: (240 + 576/Ls) reals per 5D site per H over its four passes.
 * Synchronises the stream. */
int hdcg_get_hop_profile(hdcg_t h, int prec, long long* launches, double* total_ms, double* bytes,
                         double* op_bytes);
/* Device time (ms, CUDA events) spent since profiling was enabled in each solve
 * phase: ms[0] outer-precision H applies, ms[1] preconditioner H applies (M_IRS
 * and r - H z), ms[2] FP64 true-residual H applies, ms[3] coarse CG, ms[4]
 * restriction and prolongation, ms[5] whole solves.  Synchronises the stream. */
int hdcg_get_phase_profile(hdcg_t h, double ms[6]);
/* The tensor-core stencil runs as a persistent kernel with two CTAs per SM
 * (96 KB pipeline ring each) or one (192 KB ring).  By default (0) the first
 * apply of each operator to a given number of right-hand sides times both and
 * keeps the faster; 1 or 2 forces one.  Both run the same MMAs in the same
 * order, so the results are identical.  HDCG_ERR_ARG outside 0..2. */
int hdcg_set_coarse_tc_shape(hdcg_t h, int ctas_per_sm);

/* Measurement: the mean device time (microseconds, CUDA events on the
 * handle's stream) of one tensor-core little Dirac stencil apply (k_capply_tc,
 * Sec. 5.1) of the level-1 operator to nrhs (1..16) Gaussian coarse vectors,
 * after 3 warm-up launches, over reps launches.  HDCG_ERR_ARG unless A is FP16
 * or FP32 with Nvec <= 64.  Synchronous. */
int hdcg_time_coarse_apply(hdcg_t h, int nrhs, int reps, double* us_per_apply);

/* The fine operator's hop passes come in variants: 0-2 scalar FP32 arithmetic
 * with register budgets for 1, 2 and 3 resident CTAs per SM; 3 all eight
 * neighbours prefetched (16-bit storage) or double-float arithmetic (FP64
 * storage); 4 and 5 packed FP32 (f32x2) arithmetic with the links staged in
 * shared memory (FP32 and 16-bit storage; measured slower than 0-3, and
 * rounding differently, so only run when forced).  By default (variant -1)
 * the first launch of each pass times variants 0-3 and keeps the fastest
 * (0-2 and the 16-bit variant 3 give identical bits; for FP64 storage
 * variant 3's double-float arithmetic agrees with FP64 to about 1e-14); 0..5
 * forces one (for FP64 storage variants 4 and 5 fall back to 0).
 * HDCG_ERR_ARG outside -1..5. */
int hdcg_set_hop_variant(hdcg_t h, int variant);

/* Count of library kernel launches issued on the handle since creation. */
long long hdcg_launch_count(hdcg_t h);

const char* hdcg_last_error(hdcg_t h);
void hdcg_destroy(hdcg_t h);
int hdcg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* HDCG_H */
