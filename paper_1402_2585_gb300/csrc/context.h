// Internal state of one HDCG handle (host side).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <string>
#include <vector>

#include "../../include/hdcg.h"

namespace hdcg {

// status propagation ----------------------------------------------------------
struct Error {
  int code;
  std::string msg;
};

#define HDCG_CUDA(call)                                                                   \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      throw ::hdcg::Error{HDCG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

#define HDCG_REQUIRE(cond, code, msg)                                   \
  do {                                                                  \
    if (!(cond)) throw ::hdcg::Error{(code), std::string(msg)};        \
  } while (0)

inline bool is_16bit(int prec) { return prec == HDCG_F16 || prec == HDCG_BF16 || prec == HDCG_BF16T; }
inline size_t bytes_per_real(int prec) {
  return (prec == HDCG_F64 || prec == HDCG_DF64) ? 8 : prec == HDCG_F32 ? 4 : 2;
}
// link storage slots: F64, F32, F16, BF16 (also BF16T), double-float
inline int link_slot(int prec) { return prec == HDCG_BF16T ? HDCG_BF16 : prec == HDCG_DF64 ? 4 : prec; }
constexpr int NPREC = 6;   // precision codes 0..5 (HDCG_F64 .. HDCG_DF64)

// Process-wide count of device allocations and frees.  A captured CUDA graph
// holds raw pointers; it is replayed only while this count is unchanged since
// its capture, so no buffer it may reference can have been freed or moved.
inline std::atomic<unsigned long long>& alloc_epoch_counter() {
  static std::atomic<unsigned long long> n{0};
  return n;
}
inline unsigned long long alloc_epoch() { return alloc_epoch_counter().load(); }

// device memory owned by the handle ----------------------------------------------
struct DevMem {
  void* p = nullptr;
  size_t bytes = 0;
  DevMem() = default;
  DevMem(const DevMem&) = delete;
  DevMem& operator=(const DevMem&) = delete;
  ~DevMem() { release(); }
  void release() {
    if (p) {
      cudaFree(p);
      ++alloc_epoch_counter();
    }
    p = nullptr;
    bytes = 0;
  }
  void ensure(size_t n) {
    if (bytes >= n && p) return;
    release();
    if (n == 0) return;
    cudaError_t e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
      p = nullptr;
      (void)cudaGetLastError();
      throw Error{HDCG_ERR_OOM, "cudaMalloc of " + std::to_string(n) + " bytes failed"};
    }
    ++alloc_epoch_counter();
    bytes = n;
  }
  template <typename T> T* as() const { return reinterpret_cast<T*>(p); }
};

// a fine odd/even field in the internal chunked layout
struct FieldRef {
  uint4* p;
  int prec;
};

// Moebius coefficients of the s-direction operators (site independent, real)
struct DwfCoeffs {
  double M5 = 1.8, b = 1.0, c = 0.0, mass = 0.01;
  double alpha = 0, beta = 0;   // M_ee = alpha + beta P_s
  double minv_norm = 0;         // M_ee^-1 = minv_norm * sum_{k<Ls} r^k P_s^k
  double minv_r = 0;            // r = -beta / alpha
  double rpow[6] = {0, 0, 0, 0, 0, 0};  // r^(2^j)
};

// kernel-time profile of the fine hop kernels, per storage precision
struct HopProfile {
  bool on = false;
  std::vector<cudaEvent_t> pending;  // (start, stop) pairs, recorded on the stream
  std::vector<int> pending_prec;
  long long launches[NPREC] = {};
  double ms[NPREC] = {};
  double bytes[NPREC] = {};      // everything the launches move (fused epilogues included)
  double op_bytes[NPREC] = {};   // the operator's own bytes only
};

// solve-phase timing (CUDA events on the stream, resolved on request)
enum Phase { PH_H_OUTER = 0, PH_H_SLOPPY = 1, PH_H_F64 = 2, PH_COARSE = 3, PH_TRANSFER = 4, PH_TOTAL = 5, PH_N = 6 };
struct PhaseProfile {
  std::vector<cudaEvent_t> pending;  // (start, stop) pairs
  std::vector<int> phase;
  double ms[PH_N] = {0, 0, 0, 0, 0, 0};
};

struct Ctx;
struct Subspace;
struct Coarse;

struct Ctx {
  int dims[4] = {0, 0, 0, 0};
  int Ls = 0, lslog2 = 0;
  int apbc = 0;
  cudaStream_t stream = nullptr;
  size_t V = 0, n4 = 0, n5 = 0;     // 4D volume, sites per parity, 5D sites per parity
  bool have_gauge = false, have_dwf = false;
  DwfCoeffs co;

  DevMem nbr[2];          // int32 [n4][8]: neighbour cb index of output site x (parity p)
  DevMem links[5][2];     // per link slot (F64, F32, F16, BF16) and output parity
  DevMem scratch_f[NPREC][24]; // work fields per precision (slot roles: solver.cu; 20-23: hop autotuner)
  std::map<int, int> hop_tuned;  // (prec, pass, fused, reduction) -> chosen hop variant
  int hop_force = -1;            // >= 0: every hop launch uses this variant (hdcg_set_hop_variant)
  int tc_force = 0;              // 1, 2: the tensor-core stencil's CTAs per SM (hdcg_set_coarse_tc_shape)
  DevMem red_partials, red_ticket, scalars;
  DevMem canon_in, canon_out;  // canonical <-> internal staging

  Subspace* sub = nullptr;
  Coarse* coarse = nullptr;

  HopProfile prof;
  PhaseProfile phases;
  long long launches = 0;
  std::string err;
  void* noalloc_addr = nullptr;   // device address of the no-alloc scratch array (coarse.cu)
  int noalloc_dev = -1;           // device it was looked up on

  size_t field_bytes(int prec) const { return n5 * 24 * bytes_per_real(prec); }
  uint4* scratch(int prec, int i, int nfields = 1) {
    scratch_f[prec][i].ensure(field_bytes(prec) * nfields);
    return scratch_f[prec][i].as<uint4>();
  }
};

// ---------------------------------------------------------------------------
// fine operator (dwf.cu)
// ---------------------------------------------------------------------------
enum HopPass { PASS_A = 0, PASS_B = 1, PASS_C = 2, PASS_D = 3 };
// Epilogue of pass D: out = sD * (M_oo^dag in2 - 1/4 K^dag Dh^dag in) + lam * extra
struct HopEpi {
  double sD = 1.0;
  double lam = 0.0;
  const uint4* extra = nullptr;
  // fused CG step (see apply_mdagm_cg)
  uint4* cg_x = nullptr;
  uint4* cg_r = nullptr;
  const uint4* cg_p = nullptr;
  const double* al_num = nullptr;
  const double* al_den0 = nullptr;
  const double* al_den1 = nullptr;
  double al_lam = 0.0;
  // several right-hand sides: nrhs fields fstride granules apart, scalars per rhs
  int nrhs = 1;
  size_t fstride = 0;
  const int* mask = nullptr;
};

// device scalars: 256 slots of RMAX doubles (one per right-hand side)
constexpr int RMAX = 16;

void dwf_setup_tables(Ctx& c);
void dwf_upload_gauge(Ctx& c, const void* U, bool on_device);
void dwf_set_coeffs(Ctx& c, double M5, double b, double c_, double mass);
// one hop pass; red (may be null) receives |out|^2 (FP64)
void launch_hop(Ctx& c, int pass, int prec, const uint4* in, const uint4* in2, uint4* out,
                const HopEpi& epi, double* red_result, int accumulate);
// out = Mpc in or Mpc^dag in (uses scratch slot 0)
void apply_mpc(Ctx& c, int prec, const uint4* in, uint4* out, int dagger, double* mpc_norm2);
// out = sD * H in + lam * extra; mpc_norm2 (device double, may be null) gets |Mpc in|^2
void apply_mdagm(Ctx& c, int prec, const uint4* in, uint4* out, double* mpc_norm2,
                 double sD = 1.0, double lam = 0.0, const uint4* extra = nullptr);

// One CG step fused into H: w = H p + shift p (never stored);
// alpha = *al_num / (*pw + shift * *pp); r -= alpha w; x += alpha p;
// *pw <- |Mpc p|^2 (pass B), *rr_out <- |r|^2 (pass D).
void apply_mdagm_cg(Ctx& c, int prec, const uint4* p, double shift, uint4* x, uint4* r, const double* al_num,
                    const double* pw, const double* pp, double* rr_out, int nrhs = 1, const int* mask = nullptr);
// out_r = sD * H in_r + lam * extra_r for nrhs consecutive fields; mpc_norm2[r] = |Mpc in_r|^2
void apply_mdagm_multi(Ctx& c, int prec, int nrhs, const uint4* in, uint4* out, double* mpc_norm2, double sD,
                       double lam, const uint4* extra);

// ---------------------------------------------------------------------------
// fields and BLAS-1 (blas.cu); all reductions accumulate in FP64
// ---------------------------------------------------------------------------
void canon_to_internal(Ctx& c, const void* canon, int canon_prec, uint4* out, int prec,
                       size_t nfields = 1);
void internal_to_canon(Ctx& c, const uint4* in, int prec, void* canon, int canon_prec,
                       size_t nfields = 1);
void convert_field(Ctx& c, const uint4* in, int pin, uint4* out, int pout, size_t nfields = 1);
void zero_field(Ctx& c, uint4* f, int prec, size_t nfields = 1);
// result[0] = |a|^2
void norm2(Ctx& c, const uint4* a, int prec, size_t n_reals, double* result, int nrhs = 1);
// result[0:2] = <a, b> (complex)
void cdot(Ctx& c, const uint4* a, const uint4* b, int prec, size_t n_reals, double* result);

// A launch sequence captured once from the handle's stream and replayed as one
// CUDA graph (the launch-bound inner loops of the coarse solvers).  The key
// lists every buffer and scalar baked into the captured launches; a different
// key captures again.  Graphs are not used on the legacy default stream or
// while the caller is itself capturing that stream.
struct CapturedGraph {
  cudaGraphExec_t exec = nullptr;
  std::vector<uintptr_t> key;
  long long launches = 0;   // kernels per replay (added to the handle's count)
  CapturedGraph() = default;
  CapturedGraph(const CapturedGraph&) = delete;
  CapturedGraph& operator=(const CapturedGraph&) = delete;
  ~CapturedGraph() { reset(); }
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    key.clear();
  }
};

// key: the pointers and sizes the body uses; the allocation count is added,
// so any free or reallocation anywhere forces a fresh capture
template <typename F>
void run_captured(Ctx& c, CapturedGraph& g, const std::vector<uintptr_t>& key_in, F&& body) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (c.stream == nullptr || cudaStreamIsCapturing(c.stream, &cs) != cudaSuccess ||
      cs != cudaStreamCaptureStatusNone) {
    body();
    return;
  }
  std::vector<uintptr_t> key = key_in;
  key.push_back((uintptr_t)alloc_epoch());
  if (!g.exec || g.key != key) {
    g.reset();
    const long long l0 = c.launches;
    cudaGraph_t graph = nullptr;
    HDCG_CUDA(cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal));
    try {
      body();
    } catch (...) {
      cudaStreamEndCapture(c.stream, &graph);
      if (graph) cudaGraphDestroy(graph);
      throw;
    }
    HDCG_CUDA(cudaStreamEndCapture(c.stream, &graph));
    const cudaError_t e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    HDCG_CUDA(e);
    g.key = key;
    g.launches = c.launches - l0;
    c.launches = l0;
  }
  HDCG_CUDA(cudaGraphLaunch(g.exec, c.stream));
  c.launches += g.launches;
}

// RAII phase timer: records (start, stop) events when profiling is on
struct PhaseTimer {
  Ctx& c;
  int ph;
  cudaEvent_t e0 = nullptr;
  PhaseTimer(Ctx& c_, int ph_) : c(c_), ph(ph_) {
    if (c.prof.on) {
      cudaEventCreate(&e0);
      cudaEventRecord(e0, c.stream);
    }
  }
  ~PhaseTimer() {
    if (e0) {
      cudaEvent_t e1;
      cudaEventCreate(&e1);
      cudaEventRecord(e1, c.stream);
      c.phases.pending.push_back(e0);
      c.phases.pending.push_back(e1);
      c.phases.phase.push_back(ph);
    }
  }
};

}  // namespace hdcg
