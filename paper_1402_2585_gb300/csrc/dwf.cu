// Fine operator of the HDCG library: the red-black preconditioned Shamir /
// Moebius domain-wall operator Mpc = M_oo - M_oe M_ee^-1 M_eo and
// H = Mpc^dag Mpc (Boyle, arXiv 1402.2585, Sec. 4), with
//   M_ee = M_oo = alpha + beta P_s,  M_eo = -Dh_eo K / 2,  K = b + c P_s,
//   alpha = b (4 - M5) + 1,  beta = c (4 - M5) - 1,
//   (P_s psi)_s = P_- psi_{s+1} + P_+ psi_{s-1},  psi_{Ls} -> -m psi_0, psi_{-1} -> -m psi_{Ls-1}.
//
// H runs as four fused hop passes (each one launch):
//   A  (e <- o):  t   = K M_ee^-1 Dh_eo (K psi)
//   B  (o <- e):  chi = M_oo psi - Dh_oe t / 4                 [+ |chi|^2 in FP64]
//   C  (e <- o):  u   = M_ee^-dag K^dag Dh^dag_eo chi
//   D  (o <- e):  out = M_oo^dag chi - K^dag Dh^dag_oe u / 4   [+ optional lam * extra]
// Dh^dag is Dh with gamma_mu -> -gamma_mu.  One thread owns one 5D site; the
// Ls threads of a 4D site are consecutive lanes of one warp, so the
// s-direction operators (all polynomials in the twisted shift P_s, per
// chirality) run as warp shuffles: P_s^d is one shuffle per real, and
// M_ee^-1 = minv_norm * sum_{k<Ls} r^k P_s^k (r = -beta/alpha, P_s^Ls = -m)
// is evaluated by log2(Ls) doubling steps.  The gauge links of a 4D site are
// read once per CTA group and reused by its Ls lanes (Sec. 6.5: Ls-fold link reuse).
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "dwf_kernels.cuh"

namespace hdcg {

// ------------------------------------------------------------------------------
// tables and gauge field
// ------------------------------------------------------------------------------
struct Geom {
  int L[4];
  int parity;
  size_t n4;
};

__device__ __forceinline__ void cb_coords(const Geom& g, size_t i, int* x) {
  const int hx = g.L[0] / 2;
  size_t rest = i / hx;
  x[1] = (int)(rest % g.L[1]);
  rest /= g.L[1];
  x[2] = (int)(rest % g.L[2]);
  x[3] = (int)(rest / g.L[2]);
  const int delta = (g.parity + x[1] + x[2] + x[3]) & 1;
  x[0] = 2 * (int)(i % hx) + delta;
}

__device__ __forceinline__ size_t lex_of(const Geom& g, const int* x) {
  return (size_t)x[0] + (size_t)g.L[0] * (x[1] + (size_t)g.L[1] * (x[2] + (size_t)g.L[2] * x[3]));
}

__global__ void nbr_kernel(Geom g, int* nbr) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n4) return;
  int x[4];
  cb_coords(g, i, x);
  for (int dir = 0; dir < 8; ++dir) {
    int y[4] = {x[0], x[1], x[2], x[3]};
    const int mu = dir & 3;
    y[mu] = (y[mu] + (dir < 4 ? 1 : g.L[mu] - 1)) % g.L[mu];
    nbr[i * 8 + dir] = (int)(lex_of(g, y) >> 1);
  }
}

// links[p][i][dir][3][3]: dir < 4: U_mu(x); dir >= 4: U_mu(x - mu)^dag; the
// antiperiodic time boundary is folded in as a sign.
__global__ void link_kernel(Geom g, int apbc, const double2* __restrict__ U, double2* l64,
                            float2* l32, __half2* l16, __nv_bfloat162* lb16, float4* ldf) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n4) return;
  int x[4];
  cb_coords(g, i, x);
  for (int dir = 0; dir < 8; ++dir) {
    const int mu = dir & 3;
    int y[4] = {x[0], x[1], x[2], x[3]};
    double sign = 1.0;
    if (dir >= 4) {
      y[mu] = (y[mu] + g.L[mu] - 1) % g.L[mu];
      if (apbc && mu == 3 && x[3] == 0) sign = -1.0;
    } else {
      if (apbc && mu == 3 && x[3] == g.L[3] - 1) sign = -1.0;
    }
    const double2* src = U + (lex_of(g, y) * 4 + mu) * 9;
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) {
        double2 v = dir < 4 ? src[r * 3 + c] : src[c * 3 + r];
        if (dir >= 4) v.y = -v.y;
        v.x *= sign;
        v.y *= sign;
        const int e = r * 3 + c;
        l64[(i * 8 + dir) * 9 + e] = v;
        l32[(i * 8 + dir) * 10 + e] = make_float2((float)v.x, (float)v.y);
        l16[(i * 8 + dir) * 12 + e] = __floats2half2_rn((float)v.x, (float)v.y);
        lb16[(i * 8 + dir) * 12 + e] = __floats2bfloat162_rn((float)v.x, (float)v.y);
        const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
        ldf[(i * 8 + dir) * 9 + e] =
            make_float4(rh, __double2float_rn(v.x - (double)rh), ih, __double2float_rn(v.y - (double)ih));
      }
  }
}

static Geom geom(const Ctx& c, int parity) {
  Geom g;
  for (int i = 0; i < 4; ++i) g.L[i] = c.dims[i];
  g.parity = parity;
  g.n4 = c.n4;
  return g;
}

void dwf_setup_tables(Ctx& c) {
  for (int p = 0; p < 2; ++p) {
    c.nbr[p].ensure(c.n4 * 8 * sizeof(int));
    nbr_kernel<<<(unsigned)((c.n4 + 255) / 256), 256, 0, c.stream>>>(geom(c, p), c.nbr[p].as<int>());
    HDCG_CUDA(cudaGetLastError());
    ++c.launches;
  }
}

void dwf_upload_gauge(Ctx& c, const void* U, bool on_device) {
  const size_t canon = c.V * 4 * 9 * sizeof(double2);
  const double2* src = reinterpret_cast<const double2*>(U);
  DevMem tmp;
  if (!on_device) {
    tmp.ensure(canon);
    HDCG_CUDA(cudaMemcpyAsync(tmp.p, U, canon, cudaMemcpyHostToDevice, c.stream));
    src = tmp.as<double2>();
  }
  const size_t nl = c.n4 * 8;  // links per parity; padded to whole 16-byte granules
  for (int p = 0; p < 2; ++p) {
    c.links[HDCG_F64][p].ensure(nl * 9 * sizeof(double2));
    c.links[HDCG_F32][p].ensure(nl * 10 * sizeof(float2));
    c.links[HDCG_F16][p].ensure(nl * 12 * sizeof(__half2));
    c.links[HDCG_BF16][p].ensure(nl * 12 * sizeof(__nv_bfloat162));
    c.links[link_slot(HDCG_DF64)][p].ensure(nl * 9 * sizeof(float4));
    HDCG_CUDA(cudaMemsetAsync(c.links[HDCG_F32][p].p, 0, nl * 10 * sizeof(float2), c.stream));
    HDCG_CUDA(cudaMemsetAsync(c.links[HDCG_F16][p].p, 0, nl * 12 * sizeof(__half2), c.stream));
    HDCG_CUDA(cudaMemsetAsync(c.links[HDCG_BF16][p].p, 0, nl * 12 * sizeof(__nv_bfloat162), c.stream));
    link_kernel<<<(unsigned)((c.n4 + 255) / 256), 256, 0, c.stream>>>(
        geom(c, p), c.apbc, src, c.links[HDCG_F64][p].as<double2>(), c.links[HDCG_F32][p].as<float2>(),
        c.links[HDCG_F16][p].as<__half2>(), c.links[HDCG_BF16][p].as<__nv_bfloat162>(),
        c.links[link_slot(HDCG_DF64)][p].as<float4>());
    HDCG_CUDA(cudaGetLastError());
    ++c.launches;
  }
  HDCG_CUDA(cudaStreamSynchronize(c.stream));
  c.have_gauge = true;
}

void dwf_set_coeffs(Ctx& c, double M5, double b, double cc, double mass) {
  DwfCoeffs& k = c.co;
  k.M5 = M5;
  k.b = b;
  k.c = cc;
  k.mass = mass;
  k.alpha = b * (4.0 - M5) + 1.0;
  k.beta = cc * (4.0 - M5) - 1.0;
  HDCG_REQUIRE(std::fabs(k.alpha) > 1e-300, HDCG_ERR_ARG, "b (4 - M5) + 1 must be nonzero");
  k.minv_r = -k.beta / k.alpha;
  const double denom = k.alpha * (1.0 + mass * std::pow(k.minv_r, c.Ls));
  HDCG_REQUIRE(std::fabs(denom) > 1e-300 && std::isfinite(denom), HDCG_ERR_ARG, "M_ee is singular");
  k.minv_norm = 1.0 / denom;
  double r = k.minv_r;
  for (int j = 0; j < 6; ++j) {
    k.rpow[j] = r;
    r = r * r;
  }
  c.have_dwf = true;
}

// ------------------------------------------------------------------------------
// launches
// ------------------------------------------------------------------------------
static double hop_bytes(const Ctx& c, int pass, int prec, bool extra) {
  const double fb = (double)bytes_per_real(prec);
  const double lb = (double)bytes_per_real(prec);  // link reals stored in the field precision
  double reals_field = 48.0 + ((pass == PASS_B || pass == PASS_D) ? 24.0 : 0.0) + (extra ? 24.0 : 0.0);
  return (double)c.n5 * (reals_field * fb + 8.0 * 18.0 * lb / c.Ls);
}

static void dispatch_hop(int prec, int v, int pass, bool mob, const HopArgs& a, dim3 grid, cudaStream_t st) {
  switch (prec) {
    case HDCG_F64: launch_hop_f64(v, pass, mob, a, grid, st); break;
    case HDCG_F32: launch_hop_f32(v, pass, mob, a, grid, st); break;
    case HDCG_F16: launch_hop_f16(v, pass, mob, a, grid, st); break;
    case HDCG_BF16: launch_hop_bf16(v, pass, mob, a, grid, st); break;
    case HDCG_BF16T: launch_hop_bf16t(v, pass, mob, a, grid, st); break;
    case HDCG_DF64: launch_hop_df(v, pass, mob, a, grid, st); break;
    default: throw Error{HDCG_ERR_ARG, "unknown precision code"};
  }
}

// Hop autotuner: the first launch of a (precision, pass, fused-CG) combination
// times every register-budget variant on scratch fields (never on the
// caller's data, so in-place CG updates are not repeated) and keeps the fastest.
static int hop_variant(Ctx& c, int prec, int pass, bool mob, const HopArgs& a, dim3 grid) {
  const int key = ((prec * 4 + pass) * 2 + (a.cg_r ? 1 : 0)) * 2 + (a.do_red ? 1 : 0);
  if (c.hop_force >= 0) {
    // a forced variant (hdcg_set_hop_variant); the packed variants exist for
    // FP32 and 16-bit storage only
    const bool wide = prec == HDCG_F64 || prec == HDCG_DF64;
    return (wide && c.hop_force >= 4) ? 0 : c.hop_force;
  }
  auto it = c.hop_tuned.find(key);
  if (it != c.hop_tuned.end()) return it->second;
  // scratch copies: inputs are whatever the scratch slots hold (only timing matters)
  HopArgs t = a;
  t.fstride = 0;
  t.al_mask = nullptr;
  grid.y = 1;
  uint4* s0 = c.scratch(prec, 20);
  uint4* s1 = c.scratch(prec, 21);
  uint4* s2 = c.scratch(prec, 22);
  uint4* s3 = c.scratch(prec, 23);
  HDCG_CUDA(cudaMemsetAsync(s0, 0, c.field_bytes(prec), c.stream));
  HDCG_CUDA(cudaMemsetAsync(s1, 0, c.field_bytes(prec), c.stream));
  HDCG_CUDA(cudaMemsetAsync(s2, 0, c.field_bytes(prec), c.stream));
  HDCG_CUDA(cudaMemsetAsync(s3, 0, c.field_bytes(prec), c.stream));
  t.in = s0;
  t.in2 = s1;
  t.extra = a.extra ? s1 : nullptr;
  t.out = s2;
  if (a.cg_r) {
    t.cg_r = s2;
    t.cg_x = s3;
    t.cg_p = s0;
  }
  if (a.do_red) t.red.result = c.scalars.as<double>() + 250 * RMAX;
  cudaEvent_t e0, e1;
  HDCG_CUDA(cudaEventCreate(&e0));
  HDCG_CUDA(cudaEventCreate(&e1));
  int best = 0;
  float best_ms = 1e30f;
  // variants 0-3 only: the packed variants (4, 5) round differently, and a
  // timing-dependent pick among them would make two handles' results differ
  // in the last bits; they are slower on every measured lattice anyway and
  // run only when forced
  const int nv = 4;
  for (int v = 0; v < nv; ++v) {
    dispatch_hop(prec, v, pass, mob, t, grid, c.stream);  // warm-up
    HDCG_CUDA(cudaEventRecord(e0, c.stream));
    for (int r = 0; r < 3; ++r) dispatch_hop(prec, v, pass, mob, t, grid, c.stream);
    HDCG_CUDA(cudaEventRecord(e1, c.stream));
    HDCG_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    HDCG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best_ms) {
      best_ms = ms;
      best = v;
    }
  }
  HDCG_CUDA(cudaGetLastError());
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c.launches += 4 * nv;
  c.hop_tuned[key] = best;
  // the timing fields are temporary: give their memory back (3.2 GB each for a
  // 32^3 x 64 x 16 FP64 field)
  for (int i = 20; i < 24; ++i) c.scratch_f[prec][i].release();
  return best;
}

void launch_hop(Ctx& c, int pass, int prec, const uint4* in, const uint4* in2, uint4* out,
                const HopEpi& epi, double* red_result, int accumulate) {
  HDCG_REQUIRE(c.have_gauge && c.have_dwf, HDCG_ERR_STATE, "gauge field and DWF parameters required");
  const int out_par = (pass == PASS_A || pass == PASS_C) ? 0 : 1;
  HopArgs a;
  a.in = in;
  a.in2 = in2;
  a.extra = epi.extra;
  a.out = out;
  a.links = c.links[link_slot(prec)][out_par].p;
  a.nbr = c.nbr[out_par].as<int>();
  a.n5 = c.n5;
  a.Ls = c.Ls;
  a.lslog2 = c.lslog2;
  a.b = c.co.b;
  a.c = c.co.c;
  a.alpha = c.co.alpha;
  a.beta = c.co.beta;
  a.mass = c.co.mass;
  a.minv_norm = c.co.minv_norm;
  for (int j = 0; j < 6; ++j) a.rpow[j] = c.co.rpow[j];
  a.sD = epi.sD;
  a.lam = epi.lam;
  a.fb = (float)a.b;
  a.fc = (float)a.c;
  a.falpha = (float)a.alpha;
  a.fbeta = (float)a.beta;
  a.fmass = (float)a.mass;
  a.fminv_norm = (float)a.minv_norm;
  for (int j = 0; j < 6; ++j) a.frpow[j] = (float)a.rpow[j];
  a.fsD = (float)a.sD;
  a.flam = (float)a.lam;
  a.cg_x = epi.cg_x;
  a.cg_r = epi.cg_r;
  a.cg_p = epi.cg_p;
  a.al_num = epi.al_num;
  a.al_den0 = epi.al_den0;
  a.al_den1 = epi.al_den1;
  a.al_lam = epi.al_lam;
  a.fstride = epi.nrhs > 1 ? epi.fstride : 0;
  a.al_mask = epi.mask;
  const unsigned grid = (unsigned)((c.n5 + 255) / 256);
  HDCG_REQUIRE(epi.nrhs >= 1 && epi.nrhs <= RMAX, HDCG_ERR_ARG, "1 <= right-hand sides <= 16");
  a.do_red = red_result != nullptr;
  if (a.do_red) {
    c.red_partials.ensure((size_t)grid * 4 * epi.nrhs * sizeof(double));
    a.red.partials = c.red_partials.as<double>();
    a.red.ticket = c.red_ticket.as<unsigned>();
    a.red.result = red_result;
    a.red.accumulate = accumulate;
    a.red.result_stride = 1;
  }
  const bool mob = c.co.c != 0.0;
  const dim3 grid2(grid, (unsigned)epi.nrhs);
  const int v = hop_variant(c, prec, pass, mob, a, grid2);
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (c.prof.on) {
    HDCG_CUDA(cudaEventCreate(&ev0));
    HDCG_CUDA(cudaEventCreate(&ev1));
    HDCG_CUDA(cudaEventRecord(ev0, c.stream));
  }
  dispatch_hop(prec, v, pass, mob, a, grid2, c.stream);
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
  if (c.prof.on) {
    HDCG_CUDA(cudaEventRecord(ev1, c.stream));
    c.prof.pending.push_back(ev0);
    c.prof.pending.push_back(ev1);
    c.prof.pending_prec.push_back(prec);
    c.prof.op_bytes[prec] += epi.nrhs * hop_bytes(c, pass, prec, false);
    c.prof.bytes[prec] += epi.nrhs * (hop_bytes(c, pass, prec, epi.extra != nullptr) +
                                      (epi.cg_r ? (double)c.n5 * 24 * bytes_per_real(prec) * (epi.extra ? 4.0 : 5.0)
                                                : 0.0));
  }
}

void apply_mpc(Ctx& c, int prec, const uint4* in, uint4* out, int dagger, double* mpc_norm2) {
  uint4* t = c.scratch(prec, 0);
  if (!dagger) {
    launch_hop(c, PASS_A, prec, in, nullptr, t, HopEpi{}, nullptr, 0);
    launch_hop(c, PASS_B, prec, t, in, out, HopEpi{}, mpc_norm2, 0);
  } else {
    launch_hop(c, PASS_C, prec, in, nullptr, t, HopEpi{}, nullptr, 0);
    launch_hop(c, PASS_D, prec, t, in, out, HopEpi{}, nullptr, 0);
  }
}

void apply_mdagm_cg(Ctx& c, int prec, const uint4* p, double shift, uint4* x, uint4* r, const double* al_num,
                    const double* pw, const double* pp, double* rr_out, int nrhs, const int* mask) {
  uint4* t = c.scratch(prec, 0, nrhs);
  uint4* chi = c.scratch(prec, 1, nrhs);
  HopEpi m;
  m.nrhs = nrhs;
  m.fstride = c.field_bytes(prec) / 16;
  launch_hop(c, PASS_A, prec, p, nullptr, t, m, nullptr, 0);
  launch_hop(c, PASS_B, prec, t, p, chi, m, const_cast<double*>(pw), 0);
  launch_hop(c, PASS_C, prec, chi, nullptr, t, m, nullptr, 0);
  HopEpi e = m;
  e.mask = mask;
  e.lam = shift;
  e.extra = shift != 0.0 ? p : nullptr;
  e.cg_x = x;
  e.cg_r = r;
  e.cg_p = p;
  e.al_num = al_num;
  e.al_den0 = pw;
  e.al_den1 = shift != 0.0 ? pp : nullptr;
  e.al_lam = shift;
  launch_hop(c, PASS_D, prec, t, chi, nullptr, e, rr_out, 0);
}

void apply_mdagm_multi(Ctx& c, int prec, int nrhs, const uint4* in, uint4* out, double* mpc_norm2, double sD,
                       double lam, const uint4* extra) {
  uint4* t = c.scratch(prec, 0, nrhs);
  uint4* chi = c.scratch(prec, 1, nrhs);
  HopEpi m;
  m.nrhs = nrhs;
  m.fstride = c.field_bytes(prec) / 16;
  launch_hop(c, PASS_A, prec, in, nullptr, t, m, nullptr, 0);
  launch_hop(c, PASS_B, prec, t, in, chi, m, mpc_norm2, 0);
  launch_hop(c, PASS_C, prec, chi, nullptr, t, m, nullptr, 0);
  HopEpi e = m;
  e.sD = sD;
  e.lam = lam;
  e.extra = extra;
  launch_hop(c, PASS_D, prec, t, chi, out, e, nullptr, 0);
}

void apply_mdagm(Ctx& c, int prec, const uint4* in, uint4* out, double* mpc_norm2, double sD,
                 double lam, const uint4* extra) {
  uint4* t = c.scratch(prec, 0);
  uint4* chi = c.scratch(prec, 1);
  launch_hop(c, PASS_A, prec, in, nullptr, t, HopEpi{}, nullptr, 0);
  launch_hop(c, PASS_B, prec, t, in, chi, HopEpi{}, mpc_norm2, 0);
  launch_hop(c, PASS_C, prec, chi, nullptr, t, HopEpi{}, nullptr, 0);
  HopEpi e;
  e.sD = sD;
  e.lam = lam;
  e.extra = extra;
  launch_hop(c, PASS_D, prec, t, chi, out, e, nullptr, 0);
}

}  // namespace hdcg
