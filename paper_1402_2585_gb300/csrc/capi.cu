// extern "C" entry points of libhdcg (declared in include/hdcg.h).
// Every entry point validates its arguments, converts between the canonical
// ABI layouts and the internal chunked layouts, and turns exceptions into
// return codes with a one-line reason kept on the handle.
#include <cmath>
#include <cstring>
#include <string>

#include "coarse.cuh"

namespace hdcg {
int solve(Ctx& c, const void* b, void* x, int nrhs, double tol, const hdcg_params& prm, hdcg_stats* st,
          bool on_device);
void build_subspace(Ctx& c, const hdcg_subspace_params& p);
void build_subspace_rational(Ctx& c, const hdcg_subspace_params& p);
void continue_subspace(Ctx& c, const hdcg_subspace_params& p);
void promote_subspace(Ctx& c, Ctx& src, int prec);
double coarse_tc_time_us(Ctx& c, Coarse& A, int R, int reps);
void build_coarse(Ctx& c, int prec);
void prep_source(Ctx& c, const void* eta_e, const void* eta_o, void* b);
void reconstruct(Ctx& c, const void* eta_e, const void* psi_o, void* psi_e);
void set_coarse(Ctx& c, const void* A, int prec, int on_device);

static void resolve_profile(Ctx& c) {
  auto& pr = c.prof;
  if (pr.pending.empty()) return;
  HDCG_CUDA(cudaEventSynchronize(pr.pending.back()));
  for (size_t i = 0; i + 1 < pr.pending.size(); i += 2) {
    float ms = 0.f;
    HDCG_CUDA(cudaEventElapsedTime(&ms, pr.pending[i], pr.pending[i + 1]));
    const int prec = pr.pending_prec[i / 2];
    pr.ms[prec] += ms;
    pr.launches[prec] += 1;
    cudaEventDestroy(pr.pending[i]);
    cudaEventDestroy(pr.pending[i + 1]);
  }
  pr.pending.clear();
  pr.pending_prec.clear();
}

static void resolve_phases(Ctx& c) {
  auto& pp = c.phases;
  if (pp.pending.empty()) return;
  HDCG_CUDA(cudaEventSynchronize(pp.pending.back()));
  for (size_t i = 0; i + 1 < pp.pending.size(); i += 2) {
    float ms = 0.f;
    HDCG_CUDA(cudaEventElapsedTime(&ms, pp.pending[i], pp.pending[i + 1]));
    pp.ms[pp.phase[i / 2]] += ms;
    cudaEventDestroy(pp.pending[i]);
    cudaEventDestroy(pp.pending[i + 1]);
  }
  pp.pending.clear();
  pp.phase.clear();
}

static void check_prec(int prec) {
  HDCG_REQUIRE(prec >= HDCG_F64 && prec <= HDCG_BF16T, HDCG_ERR_ARG, "unknown precision code");
}
// the fine-operator calls also take the double-float code
static void check_op_prec(int prec) {
  HDCG_REQUIRE(prec >= HDCG_F64 && prec <= HDCG_DF64, HDCG_ERR_ARG, "unknown precision code");
}
static void check_ptr(const void* p, const char* what) {
  HDCG_REQUIRE(p != nullptr, HDCG_ERR_ARG, std::string(what) + " is NULL");
}
static size_t canon_field_bytes(const Ctx& c, int prec) { return c.n5 * 24 * bytes_per_real(prec); }

}  // namespace hdcg

using namespace hdcg;

#define HDCG_ENTRY(h, body)                          \
  do {                                              \
    if (!(h)) return HDCG_ERR_ARG;                  \
    Ctx& c = *reinterpret_cast<Ctx*>(h);            \
    try {                                           \
      c.err.clear();                                \
      body;                                         \
    } catch (const Error& e) {                      \
      c.err = e.msg;                                \
      return e.code;                                \
    } catch (const std::exception& e) {             \
      c.err = e.what();                             \
      return HDCG_ERR_ARG;                          \
    }                                               \
  } while (0)

extern "C" {

int hdcg_version(void) { return 1; }

int hdcg_create(hdcg_t* h, const int dims[4], int Ls, int antiperiodic_t, void* cuda_stream) {
  if (!h || !dims) return HDCG_ERR_ARG;
  *h = nullptr;
  for (int mu = 0; mu < 4; ++mu)
    if (dims[mu] < 2 || dims[mu] % 2) return HDCG_ERR_ARG;
  if (Ls < 2 || Ls > 32 || (Ls & (Ls - 1))) return HDCG_ERR_ARG;
  Ctx* c = new Ctx();
  try {
    for (int mu = 0; mu < 4; ++mu) c->dims[mu] = dims[mu];
    c->Ls = Ls;
    c->lslog2 = 0;
    while ((1 << c->lslog2) < Ls) ++c->lslog2;
    c->apbc = antiperiodic_t ? 1 : 0;
    c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    c->V = (size_t)dims[0] * dims[1] * dims[2] * dims[3];
    c->n4 = c->V / 2;
    c->n5 = c->n4 * Ls;
    c->scalars.ensure(256 * RMAX * sizeof(double));
    c->red_ticket.ensure(RMAX * sizeof(unsigned) * 4);
    c->red_partials.ensure(((c->n5 + 255) / 256 + 1024) * 4 * sizeof(double));
    HDCG_CUDA(cudaMemset(c->scalars.p, 0, 256 * RMAX * sizeof(double)));
    HDCG_CUDA(cudaMemset(c->red_ticket.p, 0, RMAX * sizeof(unsigned) * 4));
    dwf_setup_tables(*c);
    HDCG_CUDA(cudaStreamSynchronize(c->stream));
  } catch (const Error& e) {
    delete c;
    return e.code;
  }
  *h = reinterpret_cast<hdcg_t>(c);
  return HDCG_OK;
}

void hdcg_destroy(hdcg_t h) {
  if (!h) return;
  Ctx* c = reinterpret_cast<Ctx*>(h);
  cudaStreamSynchronize(c->stream);
  for (auto e : c->prof.pending) cudaEventDestroy(e);
  for (auto e : c->phases.pending) cudaEventDestroy(e);
  delete c->sub;
  delete c->coarse;
  delete c;
}

const char* hdcg_last_error(hdcg_t h) {
  if (!h) return "null handle";
  return reinterpret_cast<Ctx*>(h)->err.c_str();
}

int hdcg_set_dwf(hdcg_t h, double M5, double b, double cc, double mass) {
  HDCG_ENTRY(h, {
    HDCG_REQUIRE(std::isfinite(M5) && std::isfinite(b) && std::isfinite(cc) && std::isfinite(mass), HDCG_ERR_ARG,
                 "non-finite DWF parameter");
    dwf_set_coeffs(c, M5, b, cc, mass);
  });
  return HDCG_OK;
}

int hdcg_set_gauge(hdcg_t h, const void* U, int on_device) {
  HDCG_ENTRY(h, {
    check_ptr(U, "U");
    dwf_upload_gauge(c, U, on_device != 0);
  });
  return HDCG_OK;
}

int hdcg_apply_mpc(hdcg_t h, const void* in, void* out, int dagger, int prec) {
  HDCG_ENTRY(h, {
    check_ptr(in, "in");
    check_ptr(out, "out");
    check_op_prec(prec);
    HDCG_REQUIRE(in != out, HDCG_ERR_ARG, "in and out must differ");
    HDCG_REQUIRE(c.have_gauge && c.have_dwf, HDCG_ERR_STATE, "gauge field and DWF parameters required");
    c.canon_in.ensure(c.field_bytes(prec));
    c.canon_out.ensure(c.field_bytes(prec));
    canon_to_internal(c, in, prec, c.canon_in.as<uint4>(), prec);
    apply_mpc(c, prec, c.canon_in.as<uint4>(), c.canon_out.as<uint4>(), dagger, nullptr);
    internal_to_canon(c, c.canon_out.as<uint4>(), prec, out, prec);
  });
  return HDCG_OK;
}

int hdcg_apply_mdagm(hdcg_t h, const void* in, void* out, int prec, double* pHp) {
  HDCG_ENTRY(h, {
    check_ptr(in, "in");
    check_ptr(out, "out");
    check_op_prec(prec);
    HDCG_REQUIRE(in != out, HDCG_ERR_ARG, "in and out must differ");
    HDCG_REQUIRE(c.have_gauge && c.have_dwf, HDCG_ERR_STATE, "gauge field and DWF parameters required");
    c.canon_in.ensure(c.field_bytes(prec));
    c.canon_out.ensure(c.field_bytes(prec));
    canon_to_internal(c, in, prec, c.canon_in.as<uint4>(), prec);
    double* d = c.scalars.as<double>() + 200 * RMAX;
    apply_mdagm(c, prec, c.canon_in.as<uint4>(), c.canon_out.as<uint4>(), pHp ? d : nullptr);
    internal_to_canon(c, c.canon_out.as<uint4>(), prec, out, prec);
    if (pHp) {
      HDCG_CUDA(cudaMemcpyAsync(pHp, d, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
      HDCG_CUDA(cudaStreamSynchronize(c.stream));
    }
  });
  return HDCG_OK;
}

static void check_level(int level) {
  HDCG_REQUIRE(level == 1 || level == 2, HDCG_ERR_ARG, "level must be 1 (fine lattice) or 2 (coarse lattice)");
}

// stage up to three canonical complex double fields through the device when
// the caller's buffers are on the host
struct HostFields {
  Ctx& c;
  DevMem d[3];
  explicit HostFields(Ctx& c_) : c(c_) {}
  const void* in(int i, const void* p, int on_device) {
    if (on_device) return p;
    const size_t bytes = c.n5 * 12 * sizeof(double2);
    d[i].ensure(bytes);
    HDCG_CUDA(cudaMemcpyAsync(d[i].p, p, bytes, cudaMemcpyHostToDevice, c.stream));
    return d[i].p;
  }
  void* out(int i, void* p, int on_device) {
    if (on_device) return p;
    d[i].ensure(c.n5 * 12 * sizeof(double2));
    return d[i].p;
  }
  void back(int i, void* p, int on_device) {
    if (!on_device)
      HDCG_CUDA(cudaMemcpyAsync(p, d[i].p, c.n5 * 12 * sizeof(double2), cudaMemcpyDeviceToHost, c.stream));
    HDCG_CUDA(cudaStreamSynchronize(c.stream));
  }
};

int hdcg_prep_source(hdcg_t h, const void* eta_e, const void* eta_o, void* b, int on_device) {
  HDCG_ENTRY(h, {
    check_ptr(eta_e, "eta_e");
    check_ptr(eta_o, "eta_o");
    check_ptr(b, "b");
    HostFields hf(c);
    const void* e = hf.in(0, eta_e, on_device);
    const void* o = hf.in(1, eta_o, on_device);
    void* bo = hf.out(2, b, on_device);
    prep_source(c, e, o, bo);
    hf.back(2, b, on_device);
  });
  return HDCG_OK;
}

int hdcg_reconstruct(hdcg_t h, const void* eta_e, const void* psi_o, void* psi_e, int on_device) {
  HDCG_ENTRY(h, {
    check_ptr(eta_e, "eta_e");
    check_ptr(psi_o, "psi_o");
    check_ptr(psi_e, "psi_e");
    HostFields hf(c);
    const void* e = hf.in(0, eta_e, on_device);
    const void* o = hf.in(1, psi_o, on_device);
    void* pe = hf.out(2, psi_e, on_device);
    reconstruct(c, e, o, pe);
    hf.back(2, psi_e, on_device);
  });
  return HDCG_OK;
}

int hdcg_build_subspace(hdcg_t h, const hdcg_subspace_params* p) {
  HDCG_ENTRY(h, {
    check_ptr(p, "params");
    HDCG_REQUIRE(p->inv_steps >= 0 && p->inv_tol > 0 && p->inv_maxiter > 0, HDCG_ERR_ARG, "bad inverse-iteration parameters");
    const int level = p->level == 0 ? 1 : p->level;
    check_level(level);
    if (level == 1) {
      if (p->method == HDCG_SUBSPACE_RATIONAL) build_subspace_rational(c, *p);
      else if (p->method == HDCG_SUBSPACE_CONTINUE) continue_subspace(c, *p);
      else {
        HDCG_REQUIRE(p->method == HDCG_SUBSPACE_INVITER, HDCG_ERR_ARG, "unknown subspace method");
        build_subspace(c, *p);
      }
    } else {
      HDCG_REQUIRE(p->method == HDCG_SUBSPACE_INVITER, HDCG_ERR_ARG, "level 2 builds by inverse iteration");
      HDCG_REQUIRE(c.sub && c.coarse, HDCG_ERR_STATE, "a level-2 subspace needs the level-1 operator");
      level2_build_subspace(c, *c.coarse, *c.sub, *p);
    }
  });
  return HDCG_OK;
}

int hdcg_promote_subspace(hdcg_t h, hdcg_t src, int prec) {
  HDCG_ENTRY(h, {
    HDCG_REQUIRE(src != nullptr, HDCG_ERR_ARG, "src handle is NULL");
    promote_subspace(c, *reinterpret_cast<Ctx*>(src), prec);
  });
  return HDCG_OK;
}

int hdcg_set_subspace(hdcg_t h, int level, const int block[4], int nvec, int prec, const void* phi, int on_device,
                      int already_orthonormal) {
  HDCG_ENTRY(h, {
    check_ptr(block, "block");
    check_ptr(phi, "phi");
    check_level(level);
    if (level == 2) {
      HDCG_REQUIRE(c.sub && c.coarse, HDCG_ERR_STATE, "a level-2 subspace needs the level-1 operator");
      HDCG_REQUIRE(prec == HDCG_F32, HDCG_ERR_ARG, "level-2 vectors are stored in F32");
      level2_set_subspace(c, *c.coarse, *c.sub, block, nvec, phi, on_device, already_orthonormal);
      return HDCG_OK;
    }
    if (!c.sub) c.sub = new Subspace();
    subspace_init(c, *c.sub, block, nvec, prec);
    const size_t bytes = (size_t)nvec * canon_field_bytes(c, HDCG_F64);
    const void* src = phi;
    DevMem tmp;
    if (!on_device) {
      tmp.ensure(bytes);
      HDCG_CUDA(cudaMemcpyAsync(tmp.p, phi, bytes, cudaMemcpyHostToDevice, c.stream));
      src = tmp.p;
    }
    canon_to_internal(c, src, HDCG_F64, c.sub->vecs.as<uint4>(), prec, nvec);
    if (!already_orthonormal) block_orthonormalise(c, *c.sub);
    HDCG_CUDA(cudaStreamSynchronize(c.stream));
  });
  return HDCG_OK;
}

int hdcg_get_subspace(hdcg_t h, int level, void* phi_host) {
  HDCG_ENTRY(h, {
    check_ptr(phi_host, "phi");
    check_level(level);
    if (level == 2) {
      HDCG_REQUIRE(c.coarse, HDCG_ERR_STATE, "no level-2 subspace");
      level2_get_subspace(c, *c.coarse, phi_host);
      return HDCG_OK;
    }
    HDCG_REQUIRE(c.sub, HDCG_ERR_STATE, "no subspace");
    const size_t bytes = (size_t)c.sub->nvec * canon_field_bytes(c, HDCG_F64);
    DevMem tmp;
    tmp.ensure(bytes);
    internal_to_canon(c, c.sub->vecs.as<uint4>(), c.sub->prec, tmp.p, HDCG_F64, c.sub->nvec);
    HDCG_CUDA(cudaMemcpyAsync(phi_host, tmp.p, bytes, cudaMemcpyDeviceToHost, c.stream));
    HDCG_CUDA(cudaStreamSynchronize(c.stream));
  });
  return HDCG_OK;
}

int hdcg_build_coarse(hdcg_t h, int level, int prec) {
  HDCG_ENTRY(h, {
    check_level(level);
    if (level == 1) {
      build_coarse(c, prec);
    } else {
      HDCG_REQUIRE(c.coarse && c.coarse->l2, HDCG_ERR_STATE, "no level-2 subspace");
      level2_assemble(c, *c.coarse, prec);
    }
  });
  return HDCG_OK;
}

int hdcg_set_coarse(hdcg_t h, const void* A, int prec, int on_device) {
  HDCG_ENTRY(h, {
    check_ptr(A, "A");
    HDCG_REQUIRE(prec == HDCG_F64 || prec == HDCG_F32 || prec == HDCG_F16, HDCG_ERR_ARG,
                 "coarse precision must be F64, F32 or F16");
    set_coarse(c, A, prec, on_device);
  });
  return HDCG_OK;
}

int hdcg_get_coarse(hdcg_t h, int level, void* A_host) {
  HDCG_ENTRY(h, {
    check_ptr(A_host, "A");
    check_level(level);
    HDCG_REQUIRE(c.coarse, HDCG_ERR_STATE, "no coarse operator");
    if (level == 1) coarse_export(c, *c.coarse, A_host);
    else level2_export(c, *c.coarse, A_host);
  });
  return HDCG_OK;
}

int hdcg_restrict_coarse(hdcg_t h, const void* x, void* c2, int nrhs) {
  HDCG_ENTRY(h, {
    check_ptr(x, "x");
    check_ptr(c2, "c2");
    HDCG_REQUIRE(c.coarse && c.coarse->l2, HDCG_ERR_STATE, "no level-2 subspace");
    level2_restrict_canon(c, *c.coarse, nrhs, x, c2);
  });
  return HDCG_OK;
}

int hdcg_prolong_coarse(hdcg_t h, const void* c2, void* x, int nrhs) {
  HDCG_ENTRY(h, {
    check_ptr(x, "x");
    check_ptr(c2, "c2");
    HDCG_REQUIRE(c.coarse && c.coarse->l2, HDCG_ERR_STATE, "no level-2 subspace");
    level2_prolong_canon(c, *c.coarse, nrhs, c2, x);
  });
  return HDCG_OK;
}

int hdcg_restrict(hdcg_t h, const void* v, int prec, void* cv) {
  HDCG_ENTRY(h, {
    check_ptr(v, "v");
    check_ptr(cv, "c");
    check_prec(prec);
    HDCG_REQUIRE(c.sub, HDCG_ERR_STATE, "no subspace");
    const int cp = c.sub->prec == HDCG_F64 ? HDCG_F64 : HDCG_F32;
    const size_t nc = c.sub->Vc * c.sub->nvec;
    c.canon_in.ensure(c.field_bytes(prec));
    canon_to_internal(c, v, prec, c.canon_in.as<uint4>(), prec);
    DevMem tmp;
    tmp.ensure(nc * 16);
    restrict_field(c, *c.sub, c.canon_in.as<uint4>(), prec, tmp.p, cp);
    cvec_convert(c, tmp.p, cp, cv, HDCG_F64, nc);
    HDCG_CUDA(cudaStreamSynchronize(c.stream));
  });
  return HDCG_OK;
}

int hdcg_prolong(hdcg_t h, const void* cv, void* v, int prec) {
  HDCG_ENTRY(h, {
    check_ptr(v, "v");
    check_ptr(cv, "c");
    check_prec(prec);
    HDCG_REQUIRE(c.sub, HDCG_ERR_STATE, "no subspace");
    const int cp = c.sub->prec == HDCG_F64 ? HDCG_F64 : HDCG_F32;
    const size_t nc = c.sub->Vc * c.sub->nvec;
    DevMem tmp;
    tmp.ensure(nc * 16);
    cvec_convert(c, cv, HDCG_F64, tmp.p, cp, nc);
    c.canon_out.ensure(c.field_bytes(prec));
    prolong_field(c, *c.sub, tmp.p, cp, c.canon_out.as<uint4>(), prec, nullptr);
    internal_to_canon(c, c.canon_out.as<uint4>(), prec, v, prec);
    HDCG_CUDA(cudaStreamSynchronize(c.stream));
  });
  return HDCG_OK;
}

int hdcg_coarse_apply(hdcg_t h, const void* x, void* y) {
  HDCG_ENTRY(h, {
    check_ptr(x, "x");
    check_ptr(y, "y");
    HDCG_REQUIRE(c.coarse, HDCG_ERR_STATE, "no coarse operator");
    const int cp = c.coarse->vec_prec();
    const size_t nc = c.coarse->Vc * c.coarse->nvec;
    DevMem tmp;
    tmp.ensure(2 * nc * 16);
    char* xi = tmp.as<char>();
    char* yi = xi + nc * 16;
    cvec_convert(c, x, HDCG_F64, xi, cp, nc);
    coarse_apply(c, *c.coarse, xi, yi, nullptr);
    cvec_convert(c, yi, cp, y, HDCG_F64, nc);
    HDCG_CUDA(cudaStreamSynchronize(c.stream));
  });
  return HDCG_OK;
}

int hdcg_coarse_apply_multi(hdcg_t h, const void* x, void* y, int nrhs) {
  HDCG_ENTRY(h, {
    check_ptr(x, "x");
    check_ptr(y, "y");
    HDCG_REQUIRE(c.coarse, HDCG_ERR_STATE, "no coarse operator");
    HDCG_REQUIRE(nrhs >= 1 && nrhs <= RMAX, HDCG_ERR_ARG, "nrhs must be 1..16");
    coarse_apply_multi_canon(c, *c.coarse, nrhs, x, y);
  });
  return HDCG_OK;
}

int hdcg_coarse_solve(hdcg_t h, const void* b, void* x, int nrhs, double tol, int maxiter, int* iterations) {
  HDCG_ENTRY(h, {
    check_ptr(b, "b");
    check_ptr(x, "x");
    HDCG_REQUIRE(c.coarse, HDCG_ERR_STATE, "no coarse operator");
    HDCG_REQUIRE(nrhs >= 1 && nrhs <= RMAX, HDCG_ERR_ARG, "nrhs must be 1..16");
    HDCG_REQUIRE(tol > 0 && maxiter > 0, HDCG_ERR_ARG, "tol > 0 and maxiter > 0");
    const int it = coarse_solve_canon(c, *c.coarse, nrhs, b, x, tol, maxiter);
    if (iterations) *iterations = it;
  });
  return HDCG_OK;
}

int hdcg_set_coarse_preconditioner(hdcg_t h, int order, double lo, double hi, double shift, double* interval) {
  HDCG_ENTRY(h, {
    HDCG_REQUIRE(c.coarse, HDCG_ERR_STATE, "no coarse operator");
    HDCG_REQUIRE(order >= 0 && order <= 256, HDCG_ERR_ARG, "order must be 0..256");
    HDCG_REQUIRE(std::isfinite(lo) && std::isfinite(hi) && std::isfinite(shift), HDCG_ERR_ARG, "non-finite argument");
    qtrunc_setup(c, *c.coarse, order, lo, hi, shift);
    if (interval) {
      interval[0] = c.coarse->qt.lo;
      interval[1] = c.coarse->qt.hi;
    }
  });
  return HDCG_OK;
}

int hdcg_coarse_precondition(hdcg_t h, const void* x, void* y, int nrhs) {
  HDCG_ENTRY(h, {
    check_ptr(x, "x");
    check_ptr(y, "y");
    HDCG_REQUIRE(c.coarse, HDCG_ERR_STATE, "no coarse operator");
    qtrunc_precondition_canon(c, *c.coarse, nrhs, x, y);
  });
  return HDCG_OK;
}

int hdcg_build_coarse_deflation(hdcg_t h, const hdcg_ldop_params* p) {
  HDCG_ENTRY(h, {
    check_ptr(p, "params");
    HDCG_REQUIRE(c.coarse, HDCG_ERR_STATE, "no coarse operator");
    ldop_build(c, *c.coarse, *p);
  });
  return HDCG_OK;
}

int hdcg_get_coarse_deflation(hdcg_t h, double* lam_host, void* Z_host) {
  HDCG_ENTRY(h, {
    check_ptr(lam_host, "lam");
    HDCG_REQUIRE(c.coarse, HDCG_ERR_STATE, "no coarse operator");
    ldop_export(c, *c.coarse, lam_host, Z_host);
  });
  return HDCG_OK;
}

int hdcg_dense_heev(int n, const double* H, double* w, double* V) {
  if (n < 1 || n > 4096 || !H || !w) return HDCG_ERR_ARG;
  try {
    dense_heev(n, H, w, V);
  } catch (...) {
    return HDCG_ERR_OOM;
  }
  return HDCG_OK;
}

int hdcg_coarse_apply_noalloc(hdcg_t h, const void* x, void* y) {
  HDCG_ENTRY(h, {
    check_ptr(x, "x");
    check_ptr(y, "y");
    HDCG_REQUIRE(c.coarse, HDCG_ERR_STATE, "no coarse operator");
    coarse_apply_noalloc(c, *c.coarse, x, y);
  });
  return HDCG_OK;
}

void hdcg_default_params(hdcg_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->algorithm = HDCG_ALG_ADEF2;
  p->outer_prec = HDCG_F32;
  p->sloppy_prec = HDCG_F32;
  p->mirs_iter = 7;
  p->mirs_shift = 1.0;
  p->coarse_tol = 0.04;
  p->coarse_maxiter = 1000;
  p->flexible = 1;
  p->maxiter = 10000;
  p->reliable_delta = 0.01;
  p->batch = 1;
  p->sloppy_codec = 0;
  p->smoother = HDCG_SMOOTHER_MIRS;
  p->cheb_order = 16;
  p->cheb_lo = 0.5;
  p->cheb_hi = 45.0;
}

int hdcg_solve(hdcg_t h, const void* b, void* x, int nrhs, double tol, const hdcg_params* p, hdcg_stats* st,
               int on_device) {
  HDCG_ENTRY(h, {
    check_ptr(b, "b");
    check_ptr(x, "x");
    hdcg_params prm;
    if (p) prm = *p;
    else hdcg_default_params(&prm);
    HDCG_REQUIRE(prm.algorithm >= HDCG_ALG_CG && prm.algorithm <= HDCG_ALG_ADEF2_FAMILY, HDCG_ERR_ARG,
                 "unknown algorithm");
    HDCG_REQUIRE(prm.maxiter > 0 && prm.reliable_delta > 0 && prm.reliable_delta < 1, HDCG_ERR_ARG,
                 "bad iteration parameters");
    HDCG_REQUIRE(prm.mirs_iter >= 1 && prm.coarse_tol > 0 && prm.coarse_maxiter > 0, HDCG_ERR_ARG,
                 "bad preconditioner parameters");
    check_prec(prm.sloppy_prec);
    hdcg_stats local;
    hdcg_stats* s = st ? st : &local;
    return solve(c, b, x, nrhs, tol, prm, s, on_device != 0);
  });
  return HDCG_ERR_ARG;  // not reached
}

int hdcg_get_phase_profile(hdcg_t h, double ms[6]) {
  HDCG_ENTRY(h, {
    check_ptr(ms, "ms");
    resolve_phases(c);
    for (int i = 0; i < PH_N; ++i) ms[i] = c.phases.ms[i];
  });
  return HDCG_OK;
}

int hdcg_set_profiling(hdcg_t h, int on) {
  HDCG_ENTRY(h, {
    resolve_profile(c);
    resolve_phases(c);
    if (on)
      for (int i = 0; i < PH_N; ++i) c.phases.ms[i] = 0;
    c.prof.on = on != 0;
    if (on) {
      for (int i = 0; i < NPREC; ++i) {
        c.prof.launches[i] = 0;
        c.prof.ms[i] = 0;
        c.prof.bytes[i] = 0;
        c.prof.op_bytes[i] = 0;
      }
    }
  });
  return HDCG_OK;
}

int hdcg_get_hop_profile(hdcg_t h, int prec, long long* launches, double* total_ms, double* bytes,
                         double* op_bytes) {
  HDCG_ENTRY(h, {
    check_op_prec(prec);
    resolve_profile(c);
    if (launches) *launches = c.prof.launches[prec];
    if (total_ms) *total_ms = c.prof.ms[prec];
    if (bytes) *bytes = c.prof.bytes[prec];
    if (op_bytes) *op_bytes = c.prof.op_bytes[prec];
  });
  return HDCG_OK;
}

int hdcg_set_coarse_tc_shape(hdcg_t h, int ctas_per_sm) {
  HDCG_ENTRY(h, {
    HDCG_REQUIRE(ctas_per_sm >= 0 && ctas_per_sm <= 2, HDCG_ERR_ARG, "ctas_per_sm must be 0, 1 or 2");
    c.tc_force = ctas_per_sm;
  });
  return HDCG_OK;
}

int hdcg_time_coarse_apply(hdcg_t h, int nrhs, int reps, double* us_per_apply) {
  HDCG_ENTRY(h, {
    check_ptr(us_per_apply, "us_per_apply");
    HDCG_REQUIRE(c.coarse, HDCG_ERR_STATE, "no coarse operator");
    *us_per_apply = coarse_tc_time_us(c, *c.coarse, nrhs, reps);
  });
  return HDCG_OK;
}

int hdcg_encode_i8(hdcg_t h, const void* in, void* scale, void* q, int nfields) {
  HDCG_ENTRY(h, {
    check_ptr(in, "in");
    check_ptr(scale, "scale");
    check_ptr(q, "q");
    HDCG_REQUIRE(nfields >= 1, HDCG_ERR_ARG, "nfields >= 1");
    encode_i8(c, in, scale, q, nfields);
  });
  return HDCG_OK;
}

int hdcg_decode_i8(hdcg_t h, const void* scale, const void* q, void* out, int nfields) {
  HDCG_ENTRY(h, {
    check_ptr(out, "out");
    check_ptr(scale, "scale");
    check_ptr(q, "q");
    HDCG_REQUIRE(nfields >= 1, HDCG_ERR_ARG, "nfields >= 1");
    decode_i8(c, scale, q, out, nfields);
  });
  return HDCG_OK;
}

int hdcg_set_hop_variant(hdcg_t h, int variant) {
  HDCG_ENTRY(h, {
    HDCG_REQUIRE(variant >= -1 && variant <= 5, HDCG_ERR_ARG, "hop variant must be -1..5");
    c.hop_force = variant;
  });
  return HDCG_OK;
}

long long hdcg_launch_count(hdcg_t h) {
  if (!h) return -1;
  return reinterpret_cast<Ctx*>(h)->launches;
}

}  // extern "C"
