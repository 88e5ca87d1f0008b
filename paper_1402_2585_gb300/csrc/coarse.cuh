// Blocked subspace and little Dirac operator state (coarse.cu).
#pragma once

#include "blas.cuh"

namespace hdcg {

struct Subspace {
  int block[4] = {0, 0, 0, 0};
  int cdims[4] = {0, 0, 0, 0};
  size_t Vc = 0;            // coarse sites (blocks)
  int nvec = 0;
  int prec = HDCG_F32;      // storage precision of the vectors
  int spb = 0;              // odd 4D sites per block
  DevMem vecs;              // nvec fields, chunked layout, precision prec
  DevMem block_of_site;     // int32 [n4]: block of each odd cb site
  DevMem block_sites;       // int32 [Vc][spb]: odd cb sites of each block, ascending
  DevMem block_coords;      // int32 [Vc][4]
  size_t vec_bytes(const Ctx& c) const { return c.field_bytes(prec); }
  uint4* vec(const Ctx& c, int k) const {
    return reinterpret_cast<uint4*>(reinterpret_cast<char*>(vecs.p) + (size_t)k * vec_bytes(c));
  }
};

// blocked second coarsening of the little Dirac operator (level2.cu): Sec. 2's
// construction on the coarse lattice; vectors FP32, A2 FP64, its inverse dense
struct Level2 {
  int block[4] = {0, 0, 0, 0};   // level-2 block extents (coarse sites)
  int cdims[4] = {0, 0, 0, 0};   // level-2 lattice extents
  size_t Vc2 = 0;                // level-2 sites
  int nvec = 0;                  // Nvec2
  int spb = 0;                   // coarse sites per level-2 block
  size_t Vc1 = 0;                // coarse sites of the operator it was built for
  int n1 = 0;                    // and its Nvec
  DevMem phi;                    // [nvec][Vc1 * n1] complex float, block-orthonormal
  DevMem blk_of_site;            // int32 [Vc1]
  DevMem sites;                  // int32 [Vc2][spb], ascending
  DevMem coords;                 // int32 [Vc2][4]
  DevMem cnbr2;                  // int32 [Vc2][81]
  DevMem A2;                     // [Vc2][81][j][k] complex double (canonical)
  DevMem Ainv;                   // dense [N2][N2] inverse of A2, N2 = Vc2 * nvec (inv_prec)
  int inv_prec = HDCG_F32;
  bool have_A2 = false;
  DevMem work, ctl;              // level-1 solver vectors and control block
  int last_iters = 2;
  int last_broke = 0;            // the last level-1 solve stopped a right-hand side on a breakdown
  CapturedGraph graph;
};

// high-mode preconditioner of the little Dirac operator (qtrunc.cu): a
// Chebyshev polynomial of the 9-block truncation Q_trunc of A (Sec. 5.2)
struct QTrunc {
  int order = 0;            // 0: none (M = 1)
  int nq = 0;               // kept blocks per coarse site (<= 9)
  double lo = 0, hi = 0, shift = 0;
  DevMem A9;                // [Vc][9][k][j] complex float (the kept blocks of A)
  DevMem nb9;               // int32 [Vc][9]
  DevMem work;              // Chebyshev vectors
};

struct Coarse {
  int prec = HDCG_F32;      // storage of A (F64, F32 or F16); vectors: F64 if A is F64 else F32
  int nvec = 0;
  size_t Vc = 0;
  DevMem A;                 // [Vc][81][k][j] complex (blocks stored transposed)
  DevMem cnbr;              // int32 [Vc][81]: coarse neighbour a + delta_l
  DevMem work;              // coarse CG vectors
  DevMem ctl;               // coarse CG control block (doubles + ints)
  DevMem qvec;              // restriction / coarse solution vectors of Q
  int last_iters = 8;
  // tensor-core form (FP16 A only): A re-tiled for tcgen05, the B tiles of the
  // current vectors, and a small state block (wait-timeout flags, per-rhs max|x|)
  DevMem Atc, xtc, tcs, sexp;
  bool tc_ready = false;
  CapturedGraph graph_cg, graph_ad1;   // captured iteration pairs of the coarse solvers
  int tc_choice = -1;       // single right-hand side: -1 undecided, 0 CUDA cores, 1 tensor cores
  int tc_cfg[RMAX + 1] = {};  // tensor-core apply to R vectors: CTAs per SM (1 or 2), 0 undecided
  // second-level (global) deflation space of A, prediagonalised: Z^dag A Z = diag(lam)
  struct Defl {
    int nd = 0;
    DevMem Z;               // [nd][Vc*Nvec] complex float
    DevMem W;               // [nd][Vc*Nvec] complex float: Z - A Z
    DevMem lam;             // [nd] double
    std::vector<double> lam_h;   // +inf marks a pair dropped from Q (non-positive or ~0)
    int dropped = 0;
  } defl;
  // an FP16 operator keeps an FP32 copy (same layout as A) from which the
  // level-2 operator is contracted
  DevMem Aacc;
  Level2* l2 = nullptr;
  QTrunc qt;
  Coarse() = default;
  Coarse(const Coarse&) = delete;
  Coarse& operator=(const Coarse&) = delete;
  ~Coarse() { delete l2; }
  int vec_prec() const { return prec == HDCG_F64 ? HDCG_F64 : HDCG_F32; }
  size_t vec_bytes() const { return Vc * nvec * (vec_prec() == HDCG_F64 ? 16 : 8); }
};

// tensor-core coarse operator (coarse_tc.cu) ---------------------------------------
struct TcState {
  unsigned err;             // bit flags of expired pipeline waits
  unsigned pad[3];
  unsigned xmax[RMAX];      // per right-hand side max(|Re x|, |Im x|) as float bits
};
struct TcGeom {
  int sites, MS, Kp, Rp, NS, NMMA, ncols, stages, parts;
  // one FP16 part of one block of A: a_gbytes stored (and copied per stage),
  // a_sbytes its shared-memory slot; lbo_a / sbo_a the distances between core
  // matrices adjacent in K / in M; rows, kgs the stored row count and 8-wide
  // K groups
  uint32_t a_gbytes, a_sbytes, lbo_a, sbo_a, b_bytes, stage_bytes, copy_bytes;
  int rows, kgs;
};
// ring_bytes: the shared-memory pipeline of one CTA (two CTAs per SM: 96 KB; one: 192 KB)
TcGeom tc_geom(int nvec, int R, int parts, uint32_t ring_bytes = 96 * 1024);
bool coarse_tc_supported(const Coarse& A);
void coarse_tc_prepare(Ctx& c, Coarse& A);
// coarse CG on R right-hand sides (FP32 vectors [a][k][r]) with the tensor-core operator
int coarse_cg_tc(Ctx& c, Coarse& A, int R, const void* rhs, void* sol, double tol, int maxiter,
                 double shift = 0.0);
// building blocks of the tensor-core apply (x, y FP32 [a][k][r]; xmax per-rhs max|x| bits)
void coarse_tc_max(Ctx& c, const float2* x, size_t ne, int R, unsigned* xmax);
void coarse_tc_to_b(Ctx& c, Coarse& A, int R, const float2* x, const unsigned* xmax, const int* skip);
void coarse_tc_apply(Ctx& c, Coarse& A, int R, const float2* x, float2* y, const unsigned* xmax, const int* skip,
                     double* dot_result, double shift);
void coarse_tc_check(Ctx& c, Coarse& A);
// Y = A X, x and y canonical [R][Vc][Nvec] complex double (device); F16 A on the tensor cores
void coarse_apply_multi_canon(Ctx& c, Coarse& A, int R, const void* x64, void* y64);
// coarse solve A x = b for R right-hand sides, b and x canonical [R][Vc][Nvec] complex
// double (device); A-DEF1 when a deflation space exists, else CG; returns iterations
int coarse_solve_canon(Ctx& c, Coarse& A, int R, const void* b64, void* x64, double tol, int maxiter);
// single right-hand side: time both coarse apply paths once and keep the faster
bool coarse_use_tc_single(Ctx& c, Coarse& A);

// [R][ne] complex double (canonical) <-> [ne][R] complex float (device, asynchronous)
void coarse_canon_to_multi(Ctx& c, const void* in64, float2* out, size_t ne, int R);
void coarse_multi_to_canon(Ctx& c, const float2* in, void* out64, size_t ne, int R);

// blocked second coarsening (level2.cu)
void level2_init(Ctx& c, Coarse& A, const Subspace& s, const int block[4], int nvec);
void level2_build_subspace(Ctx& c, Coarse& A, const Subspace& s, const hdcg_subspace_params& p);
void level2_set_subspace(Ctx& c, Coarse& A, const Subspace& s, const int block[4], int nvec, const void* phi,
                         int on_device, int already_orthonormal);
void level2_get_subspace(Ctx& c, const Coarse& A, void* host);
void level2_orthonormalise(Ctx& c, Level2& L);
// A2 = P2^dag A P2 and its dense inverse (stored in inv_prec: F32 or F64)
void level2_assemble(Ctx& c, Coarse& A, int inv_prec);
void level2_export(Ctx& c, const Coarse& A, void* host);
// c2 = R2 x, x = P2 c2 on canonical vectors [R][Vc][Nvec] / [R][Vc2][Nvec2] (complex double, device)
void level2_restrict_canon(Ctx& c, const Coarse& A, int R, const void* x64, void* c64);
void level2_prolong_canon(Ctx& c, const Coarse& A, int R, const void* c64, void* x64);
bool level2_active(const Coarse& A);
// level-1 solve A x = b (FP32 [e][r]) by A-DEF2 with Q2 = P2 A2^-1 R2; returns iterations
int level1_solve(Ctx& c, Coarse& A, int R, const void* rhs, void* sol, double tol, int maxiter);

// Chebyshev preconditioner of Q_trunc (qtrunc.cu): set up (order 0 removes it;
// hi <= 0: 1.1 x the power-iteration estimate of lambda_max(Q_trunc + shift);
// lo <= 0: hi |lo|, or hi / 90 for lo = 0), apply to FP32 [e][r] vectors
void qtrunc_setup(Ctx& c, Coarse& A, int order, double lo, double hi, double shift);
void qtrunc_apply(Ctx& c, const Coarse& A, int R, const float2* x, float2* y, double shift, const int* skip);
void qtrunc_precondition(Ctx& c, Coarse& A, int R, const float2* r, float2* y, unsigned* xm, const int* skip);
void qtrunc_precondition_canon(Ctx& c, Coarse& A, int R, const void* x64, void* y64);

// subspace geometry (host tables -> device)
void subspace_init(Ctx& c, Subspace& s, const int block[4], int nvec, int prec);
// Gaussian noise in every subspace vector (splitmix64 counter stream, Box-Muller),
// drawn in canonical order [k][cb][s][spin][colour][re, im]
void subspace_noise(Ctx& c, Subspace& s, uint64_t seed);
// v <- (H + shift)^-1 v by CG in precision wp, v stored in vprec (solver.cu)
void inverse_step(Ctx& c, int wp, uint4* v, int vprec, double shift, double tol, int maxiter);
// block orthonormalisation: two rounds of (block Gram matrix in FP64,
// Cholesky G = R^dag R in FP64, Phi <- Phi R^-1)
void block_orthonormalise(Ctx& c, Subspace& s);

// c[b][k] = <phi_k^b, v>; c complex in coarse vector precision (vprec)
void restrict_field(Ctx& c, const Subspace& s, const uint4* v, int vprec, void* cvec, int cprec);
// out = (add ? add : 0) + sum_k c[b(x)][k] phi_k(x)
void prolong_field(Ctx& c, const Subspace& s, const void* cvec, int cprec, uint4* out, int oprec,
                   const uint4* add);

// little Dirac operator
void coarse_init(Ctx& c, Coarse& A, const Subspace& s, int prec);
void coarse_assemble(Ctx& c, Coarse& A, const Subspace& s, int hprec);
// y = A x (+ |<x, y>| real part into red_result if not null); vectors in A.vec_prec()
void coarse_apply(Ctx& c, const Coarse& A, const void* x, void* y, double* xAx);
// coarse CG to relative residual tol from zero; returns iterations
int coarse_cg(Ctx& c, Coarse& A, const void* rhs, void* sol, double tol, int maxiter);
// coarse vectors: complex double <-> coarse vector precision (n complex)
void cvec_convert(Ctx& c, const void* in, int pin, void* out, int pout, size_t n);
// Size of the fixed device array behind the no-alloc coarse apply (32 MiB:
// up to 838,860 coarse unknowns with FP32/FP16 A, 699,050 with FP64 A).
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;
size_t coarse_apply_noalloc_bytes(const Coarse& A);
// y = A x on canonical complex double coarse vectors (device) without allocating
void coarse_apply_noalloc(Ctx& c, const Coarse& A, const void* x64, void* y64);
// several right-hand sides: coarse vectors [a][k][r]
void restrict_multi(Ctx& c, const Subspace& s, const uint4* v, int vprec, int R, void* cvec, int cprec);
// out_r = f_r (add_r + P c_r); add (may be null) in oprec or, for an FP32/FP64
// output, in FP16 (add_prec); f_r = sqrt(un_den[r] / un_num[0]) when un_num is
// given (undoes convert_scaled's unit-RMS scaling), else 1
void prolong_multi(Ctx& c, const Subspace& s, const void* cvec, int cprec, int R, uint4* out, int oprec,
                   const uint4* add, int add_prec = -1, const double* un_num = nullptr,
                   const double* un_den = nullptr);
// coarse CG on (A + shift) for R right-hand sides; with deflate and a second-level
// deflation space (and no shift) the solve is A-DEF1 instead
int coarse_cg_multi(Ctx& c, Coarse& A, int R, const void* rhs, void* sol, double tol, int maxiter,
                    double shift = 0.0, bool deflate = true);
// y partials of (A) p on the CUDA cores for a coarse FP32/FP16 operator and FP32
// vectors [a][k][r]; returns the number of partial products (consumers add them);
// per-rhs <p, A p> into pAp; nothing happens while *skip is nonzero
int coarse_apply_partials(Ctx& c, const Coarse& A, int R, const float2* p, float2* wpart, const int* skip,
                          double* pAp);
// second-level deflation of the little Dirac operator (ldop.cu)
void ldop_build(Ctx& c, Coarse& A, const hdcg_ldop_params& prm);
void ldop_export(Ctx& c, const Coarse& A, double* lam_host, void* Z_host);
// dense Hermitian eigensolver of the third level (host): H, V complex row-major n x n
void dense_heev(int n, const double* H, double* w, double* V);
int coarse_adef1(Ctx& c, Coarse& A, int R, const void* rhs, void* sol, double tol, int maxiter);
// n complex Gaussians, splitmix64 stream seed, canonical order (same stream as subspace_noise)
void coarse_noise(Ctx& c, float2* out, size_t n, uint64_t seed);
void coarse_apply_multi(Ctx& c, const Coarse& A, int R, const void* x, void* y);
// canonical import of A (complex double [Vc][81][j][k], host or device) into storage A.prec
void coarse_import(Ctx& c, Coarse& A, const void* src, int on_device);
// canonical export of A (complex double [Vc][81][j][k], host)
void coarse_export(Ctx& c, const Coarse& A, void* host);

}  // namespace hdcg
