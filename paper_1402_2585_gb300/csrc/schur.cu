// Source preparation and reconstruction of the Schur form (Sec. 4).
//
// The full domain wall system D psi = eta splits over the even and odd
// checkerboards, D = [[M_ee, M_eo], [M_oe, M_oo]] with M_ee = M_oo (s-local)
// and M_eo, M_oe = -Dh K / 2.  Its odd half solves the Schur-complement
// system Mpc psi_o = eta_o - M_oe M_ee^-1 eta_e, here through the normal
// equation H psi_o = b, b = Mpc^dag (eta_o - M_oe M_ee^-1 eta_e); the even
// half is psi_e = M_ee^-1 (eta_e - M_eo psi_o).  Both run once per solve, in
// FP64 on the canonical complex double fields.
#include "dwf_kernels.cuh"

namespace hdcg {

namespace {

// out = K M_ee^-1 in (s-local, either parity)
__global__ void k_kminv(const HopArgs a) {
  const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = gtid < a.n5;
  const size_t site5 = active ? gtid : 0;
  const int s = threadIdx.x & (a.Ls - 1);
  double v[24];
  load_spinor<f64_t, double>(a.in, site5, a.n5, v);
  apply_minv<double, false>(v, s, a);
  apply_lin<double, false>(v, a.b, a.c, s, a.Ls, a.mass);
  if (active) store_spinor<f64_t, double>(a.out, site5, a.n5, v);
}

// acc = Dh (K^KIN in) at the output parity; EPI 0: out = in2 + acc / 2,
// EPI 1: out = M_ee^-1 (in2 + acc / 2)
template <bool KIN, int EPI>
__global__ void k_hop_half(const HopArgs a) {
  const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = gtid < a.n5;
  const int s = threadIdx.x & (a.Ls - 1);
  const size_t x4 = active ? (gtid >> a.lslog2) : 0;
  const size_t site5 = x4 * a.Ls + s;
  double acc[24];
#pragma unroll
  for (int i = 0; i < 24; ++i) acc[i] = 0.0;
  const int4 nb0 = __ldg(reinterpret_cast<const int4*>(a.nbr) + x4 * 2);
  const int4 nb1 = __ldg(reinterpret_cast<const int4*>(a.nbr) + x4 * 2 + 1);
  const int nbv[8] = {nb0.x, nb0.y, nb0.z, nb0.w, nb1.x, nb1.y, nb1.z, nb1.w};
  const uint4* lk = reinterpret_cast<const uint4*>(a.links) + x4 * 8 * LinkGran<double2>::g;
  hop_pair<f64_t, double, double2, 0, 1, KIN>(a, a.in, nbv, lk, s, acc);
  hop_pair<f64_t, double, double2, 1, 1, KIN>(a, a.in, nbv, lk, s, acc);
  hop_pair<f64_t, double, double2, 2, 1, KIN>(a, a.in, nbv, lk, s, acc);
  hop_pair<f64_t, double, double2, 3, 1, KIN>(a, a.in, nbv, lk, s, acc);
  double self[24];
  load_spinor<f64_t, double>(a.in2, site5, a.n5, self);
#pragma unroll
  for (int i = 0; i < 24; ++i) acc[i] = self[i] + 0.5 * acc[i];
  if (EPI == 1) apply_minv<double, false>(acc, s, a);
  if (active) store_spinor<f64_t, double>(a.out, site5, a.n5, acc);
}

HopArgs args(const Ctx& c, int out_par) {
  HopArgs a{};
  a.links = c.links[HDCG_F64][out_par].p;
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
  a.sD = 1.0;
  return a;
}

}  // namespace

// b = Mpc^dag (eta_o - M_oe M_ee^-1 eta_e); fields canonical complex double (device)
void prep_source(Ctx& c, const void* eta_e, const void* eta_o, void* b) {
  HDCG_REQUIRE(c.have_gauge && c.have_dwf, HDCG_ERR_STATE, "gauge field and DWF parameters required");
  uint4* e = c.scratch(HDCG_F64, 2);
  uint4* o = c.scratch(HDCG_F64, 3);
  uint4* t = c.scratch(HDCG_F64, 4);
  canon_to_internal(c, eta_e, HDCG_F64, e, HDCG_F64);
  canon_to_internal(c, eta_o, HDCG_F64, o, HDCG_F64);
  const unsigned g = (unsigned)((c.n5 + 255) / 256);
  HopArgs a = args(c, 0);
  a.in = e;
  a.out = t;
  k_kminv<<<g, 256, 0, c.stream>>>(a);             // t_e = K M_ee^-1 eta_e
  a = args(c, 1);
  a.in = t;
  a.in2 = o;
  a.out = e;
  k_hop_half<false, 0><<<g, 256, 0, c.stream>>>(a);  // eta_o' = eta_o + Dh_oe t_e / 2
  HDCG_CUDA(cudaGetLastError());
  c.launches += 2;
  apply_mpc(c, HDCG_F64, e, t, 1, nullptr);         // b = Mpc^dag eta_o'
  internal_to_canon(c, t, HDCG_F64, b, HDCG_F64);
}

// psi_e = M_ee^-1 (eta_e - M_eo psi_o) = M_ee^-1 (eta_e + Dh_eo K psi_o / 2)
void reconstruct(Ctx& c, const void* eta_e, const void* psi_o, void* psi_e) {
  HDCG_REQUIRE(c.have_gauge && c.have_dwf, HDCG_ERR_STATE, "gauge field and DWF parameters required");
  uint4* e = c.scratch(HDCG_F64, 2);
  uint4* o = c.scratch(HDCG_F64, 3);
  uint4* t = c.scratch(HDCG_F64, 4);
  canon_to_internal(c, eta_e, HDCG_F64, e, HDCG_F64);
  canon_to_internal(c, psi_o, HDCG_F64, o, HDCG_F64);
  const unsigned g = (unsigned)((c.n5 + 255) / 256);
  HopArgs a = args(c, 0);
  a.in = o;
  a.in2 = e;
  a.out = t;
  k_hop_half<true, 1><<<g, 256, 0, c.stream>>>(a);
  HDCG_CUDA(cudaGetLastError());
  ++c.launches;
  internal_to_canon(c, t, HDCG_F64, psi_e, HDCG_F64);
}

}  // namespace hdcg
