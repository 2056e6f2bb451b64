// api.cu -- host runtime of libsdpgpu: instance setup, the batched group
// engine that drives Algorithm 1 (ADMM) with the LOBPCG projection of
// Algorithm 3 over any number of instances, and the C ABI of sdpgpu.h.
//
// Every arithmetic step of an iteration runs in the kernels; the host
// decides control flow (mode, LOBPCG continuation, expansion, termination)
// from small per-instance control blocks read back after each step.
#include <cuda_runtime.h>
#include <cusolverDn.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <vector>

#include "../../include/sdpgpu.h"
#include "common.cuh"
#include "kernels.h"
#include "runtime.h"
#include "prof.h"

using namespace sdpg;

#define CK(x)                                              \
  do {                                                     \
    cudaError_t e_ = (x);                                  \
    if (e_ != cudaSuccess) {                               \
      set_err(cudaGetErrorString(e_), __FILE__, __LINE__); \
      return SDP_E_CUDA;                                   \
    }                                                      \
  } while (0)

static thread_local char g_err[512];
static void set_err(const char* what, const char* file, int line) {
  snprintf(g_err, sizeof(g_err), "%s (%s:%d)", what, file, line);
}
extern "C" const char* sdp_last_error(void) { return g_err; }

static const int TPB = 256;

// Limit of every bounded device wait, in nanoseconds (0: the kernels' own
// default).  Set only by sdp_set_wait_limit, for tests of the give-up path.
static unsigned long long g_wait_limit_ns = 0;
extern "C" int sdp_set_wait_limit(double seconds) {
  if (!(seconds >= 0.0) || seconds > 60.0) return SDP_E_INVALID;
  g_wait_limit_ns = (unsigned long long)(seconds * 1e9);
  if (seconds > 0.0 && g_wait_limit_ns == 0) g_wait_limit_ns = 1;
  return SDP_OK;
}

namespace sdpg {
Prof& prof() {
  static Prof P;
  return P;
}
}  // namespace sdpg

extern "C" void sdp_prof_enable(int on) {
  prof().flush();
  prof().on = on != 0;
}
extern "C" void sdp_prof_reset(void) {
  Prof& P = prof();
  P.flush();
  for (int f = 0; f < SDP_PROF_FAMILIES; ++f) {
    P.launches[f] = P.timed[f] = 0;
    P.ms[f] = P.flops[f] = P.bytes[f] = 0.0;
  }
  P.named.clear();
}
extern "C" int sdp_prof_named(int idx, char* name, int name_cap, sdp_prof_entry* out) {
  Prof& P = prof();
  P.flush();
  if (idx < 0 || idx >= (int)P.named.size() || !out) return SDP_E_INVALID;
  auto it = P.named.begin();
  std::advance(it, idx);
  if (name && name_cap > 0) snprintf(name, (size_t)name_cap, "%s", it->first.c_str());
  out->launches = it->second.launches;
  out->ms = it->second.ms;
  out->timed = it->second.timed;
  out->flops = it->second.flops;
  out->bytes = it->second.bytes;
  return SDP_OK;
}
extern "C" int sdp_prof_get(int fam, sdp_prof_entry* out) {
  if (fam < 0 || fam >= SDP_PROF_FAMILIES || !out) return SDP_E_INVALID;
  Prof& P = prof();
  P.flush();
  out->launches = P.launches[fam];
  out->ms = P.ms[fam];
  out->timed = P.timed[fam];
  out->flops = P.flops[fam];
  out->bytes = P.bytes[fam];
  return SDP_OK;
}

// ---------------------------------------------------------------------------
// settings
// ---------------------------------------------------------------------------
extern "C" void sdp_default_settings(sdp_settings* s) {
  s->rho = 1.0;
  s->sigma = 1e-6;
  s->alpha = 1.6;
  s->eps_abs = 1e-4;
  s->eps_rel = 0.0;
  s->eps_pinf = 1e-4;
  s->eps_dinf = 1e-4;
  s->max_iter = 5000;
  s->check_every = 40;
  s->lobpcg_max_iter = 20;
  s->precision = SDP_PREC_FP64;
  s->exact_only = 0;
  s->tol_coef = 10.0;
  s->tol_exp = 1.01;
  s->expand_frac = 1.0 / 50.0;
  s->mode_frac = 1.0 / 3.0;
  s->seed = 0;
  s->rr_method = 0;
  s->rr_fp32 = 0;
  s->proj_neg = 0;
  s->exact_solver = 0;
  s->soft_lock = 0;
}

extern "C" const char* sdp_status_str(int s) {
  switch (s) {
    case SDP_OK: return "OK";
    case SDP_SOLVED: return "SOLVED";
    case SDP_PRIMAL_INFEASIBLE: return "PRIMAL_INFEASIBLE";
    case SDP_DUAL_INFEASIBLE: return "DUAL_INFEASIBLE";
    case SDP_MAX_ITER: return "MAX_ITER";
    case SDP_RUNNING: return "RUNNING";
    case SDP_QUEUED: return "QUEUED";
    case SDP_E_INVALID: return "E_INVALID";
    case SDP_E_NOMEM: return "E_NOMEM";
    case SDP_E_CUDA: return "E_CUDA";
    case SDP_E_NUMERICAL: return "E_NUMERICAL";
    case SDP_E_TIMEOUT: return "E_TIMEOUT";
    case SDP_E_STATE: return "E_STATE";
  }
  return "UNKNOWN";
}

static bool settings_ok(const sdp_settings* s) {
  return s->rho > 0 && s->sigma > 0 && s->alpha > 0 && s->alpha < 2 && s->eps_abs >= 0 && s->eps_rel >= 0 &&
         s->max_iter >= 1 && s->check_every >= 1 && s->lobpcg_max_iter >= 1 && s->precision >= 0 &&
         s->precision <= 2 && (s->rr_method == 0 || s->rr_method == 1) && (s->rr_fp32 == 0 || s->rr_fp32 == 1) && (s->proj_neg == 0 || s->proj_neg == 1) && (s->exact_solver == 0 || s->exact_solver == 1) && (s->soft_lock == 0 || s->soft_lock == 1) && s->tol_coef > 0 && s->expand_frac > 0 && s->mode_frac > 0 && s->mode_frac <= 0.5;
}

// ---------------------------------------------------------------------------
// sizes of one context's device state
// ---------------------------------------------------------------------------
static int round_up(int v, int a) { return (v + a - 1) / a * a; }

struct Layout {
  int n, ld, mc, nent, nF, mcap, pcap, bexp;
  long nnz;
  size_t gpart_elems;
};

static Layout make_layout(int n, int mc, long nnz, int nent, int nF, const sdp_settings& st) {
  Layout L;
  L.n = n;
  L.ld = round_up(n, 8);
  L.mc = mc;
  L.nnz = nnz;
  L.nent = nent;
  L.nF = nF;
  L.bexp = std::max(1, (int)ceil(st.expand_frac * n));
  L.mcap = std::min(n, (int)ceil(st.mode_frac * n) + 2 * L.bexp);
  L.pcap = 3 * L.mcap;
  size_t p2 = (size_t)L.pcap * L.pcap;
  L.gpart_elems = std::max<size_t>((size_t)1 << 22, p2);
  return L;
}

struct Alloc {
  size_t off = 0;
  template <typename T>
  size_t take(size_t count) {
    size_t o = off;
    off += (count * sizeof(T) + 255) / 256 * 256;
    return o;
  }
};

// returns total bytes and fills offsets through the lambda
static size_t layout_bytes(const Layout& L, Inst* inst, char* base) {
  Alloc a;
  size_t nn = (size_t)L.ld * L.n;
  size_t blk = (size_t)L.ld * L.pcap;
  size_t p2 = (size_t)L.pcap * L.pcap;
  int mc = std::max(L.mc, 1), ne = std::max(L.nent, 1);
  long nz = std::max<long>(L.nnz, 1);
  size_t o_C = a.take<double>(nn), o_x = a.take<double>(nn), o_Z = a.take<double>(nn), o_Y = a.take<double>(nn),
         o_W = a.take<double>(nn), o_xp = a.take<double>(nn), o_Yp = a.take<double>(nn);
  size_t o_b = a.take<double>(mc), o_ye = a.take<double>(mc), o_ze = a.take<double>(mc),
         o_yep = a.take<double>(mc), o_u = a.take<double>(mc), o_v = a.take<double>(mc), o_tv = a.take<double>(mc);
  size_t o_ei = a.take<int>(ne), o_ej = a.take<int>(ne), o_eptr = a.take<int>(ne + 1), o_econ = a.take<int>(nz);
  size_t o_eval = a.take<double>(nz), o_er = a.take<double>(ne), o_ec = a.take<double>(ne);
  size_t o_cptr = a.take<int>(mc + 1), o_cent = a.take<int>(nz), o_cw = a.take<double>(nz);
  size_t o_mask = a.take<uint32_t>((nn + 31) / 32);
  size_t o_kd = a.take<double>(mc), o_isD = a.take<int>(mc), o_fpos = a.take<int>(mc), o_Fl = a.take<int>(mc);
  // K off-diagonal CSR: sized by the caller-provided bound (stored in nnz of K later) -> reserve generously
  size_t o_kptr = a.take<int>(mc + 1);
  size_t o_kcol = 0, o_kval = 0, o_Lf = 0;
  (void)o_kcol; (void)o_kval; (void)o_Lf;
  size_t o_S0 = a.take<double>(blk), o_S1 = a.take<double>(blk), o_A0 = a.take<double>(blk),
         o_A1 = a.take<double>(blk);
  size_t o_G = a.take<double>(p2), o_M = a.take<double>(p2), o_Li = a.take<double>(p2), o_H = a.take<double>(p2),
         o_U = a.take<double>(p2);
  size_t o_Cf = a.take<double>((size_t)L.pcap * L.mcap), o_th = a.take<double>(L.pcap),
         o_rn = a.take<double>(L.pcap), o_gp = a.take<double>(L.gpart_elems), o_sl = a.take<int>(L.mcap);
  size_t o_E = a.take<double>(nn), o_EV = a.take<double>(nn), o_el = a.take<double>(2 * (size_t)L.n),
         o_er2 = a.take<double>(2 * (size_t)L.n + 2), o_eo = a.take<int>(L.n);
  size_t o_ctl = a.take<Ctl>(1), o_chk = a.take<Check>(1);
  size_t o_whi = a.take<uint16_t>(nn), o_wlo = a.take<uint16_t>(nn);
  size_t o_bhi = a.take<uint16_t>((size_t)L.ld * L.mcap), o_blo = a.take<uint16_t>((size_t)L.ld * L.mcap);
  size_t o_tcp = a.take<float>((size_t)8 * L.ld * L.mcap);
  if (inst && base) {
    memset(inst, 0, sizeof(*inst));
    inst->n = L.n; inst->ld = L.ld; inst->mc = L.mc; inst->nent = L.nent; inst->mcap = L.mcap;
    inst->bexp = L.bexp; inst->pcap = L.pcap; inst->nF = L.nF;
    inst->C = (double*)(base + o_C); inst->x = (double*)(base + o_x); inst->Z = (double*)(base + o_Z);
    inst->Y = (double*)(base + o_Y); inst->W = (double*)(base + o_W); inst->xprev = (double*)(base + o_xp);
    inst->Yprev = (double*)(base + o_Yp);
    inst->b = (double*)(base + o_b); inst->ye = (double*)(base + o_ye); inst->ze = (double*)(base + o_ze);
    inst->yeprev = (double*)(base + o_yep); inst->u = (double*)(base + o_u); inst->v = (double*)(base + o_v);
    inst->tv = (double*)(base + o_tv);
    inst->ent_i = (int*)(base + o_ei); inst->ent_j = (int*)(base + o_ej); inst->ent_ptr = (int*)(base + o_eptr);
    inst->ent_con = (int*)(base + o_econ); inst->ent_val = (double*)(base + o_eval);
    inst->ent_r = (double*)(base + o_er); inst->ent_corr = (double*)(base + o_ec);
    inst->con_ptr = (int*)(base + o_cptr); inst->con_ent = (int*)(base + o_cent); inst->con_w = (double*)(base + o_cw);
    inst->smask = (uint32_t*)(base + o_mask);
    inst->kdiag = (double*)(base + o_kd); inst->isD = (int*)(base + o_isD); inst->fpos = (int*)(base + o_fpos);
    inst->Flist = (int*)(base + o_Fl); inst->k_ptr = (int*)(base + o_kptr);
    inst->S[0] = (double*)(base + o_S0); inst->S[1] = (double*)(base + o_S1);
    inst->AS[0] = (double*)(base + o_A0); inst->AS[1] = (double*)(base + o_A1);
    inst->G = (double*)(base + o_G); inst->M = (double*)(base + o_M); inst->Linv = (double*)(base + o_Li);
    inst->H = (double*)(base + o_H); inst->U = (double*)(base + o_U);
    inst->Coef = (double*)(base + o_Cf); inst->theta = (double*)(base + o_th); inst->resn = (double*)(base + o_rn);
    inst->gpart = (double*)(base + o_gp);
    inst->slot = (int*)(base + o_sl);
    inst->E = (double*)(base + o_E); inst->EV = (double*)(base + o_EV); inst->elam = (double*)(base + o_el);
    inst->erot = (double*)(base + o_er2); inst->eord = (int*)(base + o_eo);
    inst->ctl = (Ctl*)(base + o_ctl); inst->chk = (Check*)(base + o_chk);
    inst->Whi = base + o_whi; inst->Wlo = base + o_wlo; inst->Bhi = base + o_bhi; inst->Blo = base + o_blo;
    inst->tcpart = (float*)(base + o_tcp);
  }
  return a.off;
}

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct sdp_ctx {
  sdp_settings st;
  cudaStream_t stream = nullptr;
  int device = 0;
  bool ready = false;
  Layout L{};
  Inst inst{};           // host copy of the device descriptor
  char* dmem = nullptr;  // main device allocation
  char* dK = nullptr;    // K off-diagonal entries and Schur factor
  size_t dbytes = 0, kbytes = 0;
  int proj_only = 0;     // standalone projection context (no constraints)
  // per-solve host state
  int k = 0, status = SDP_OK, finished = 0;
  int mode = MODE_EXACT, m = 0, mP = 0, nfresh = 0, cnt_pos = 0, cnt_neg = 0;
  int cert_kind = 0;
  std::vector<double> cert_y, cert_M;
  sdp_info info{};
  std::chrono::steady_clock::time_point t0;
  std::map<int, sdp_ctx*> projs;  // lazily created contexts of sdp_project_psd, by n
  void* group_cache = nullptr;  // reusable engine state of a projection context
  double proj_res_pos2 = 0.0;
  int proj_steps = 0;
  // precision ladder (mixed precision): ||W||_F^2 and the smallest |Ritz
  // value| seen by the last projection (0: unknown)
  double wfro2 = 0.0, thmin = 0.0;
  void* oz = nullptr;      // workspace of sdp_dense_product (grown on demand)
  size_t oz_bytes = 0;
  int* oz_err = nullptr;   // its wait-error flag
};

static void ctx_free(sdp_ctx* c) {
  if (c->dmem) cudaFree(c->dmem);
  if (c->dK) cudaFree(c->dK);
  if (c->oz) cudaFree(c->oz);
  if (c->oz_err) cudaFree(c->oz_err);
  c->dmem = nullptr;
  c->dK = nullptr;
  c->oz = nullptr;
  c->oz_err = nullptr;
  c->oz_bytes = 0;
  c->ready = false;
}

// grow a device workspace to at least `need` bytes (contents not kept)
static int grow_work(void** p, size_t* cap, size_t need) {
  if (*cap >= need && *p) return SDP_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  const size_t want = need + need / 8;
  if (cudaMalloc(p, want) != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return SDP_E_NOMEM;
  }
  *cap = want;
  return SDP_OK;
}

extern "C" int sdp_create(sdp_ctx** out, const sdp_settings* settings, void* stream) {
  if (!out) return SDP_E_INVALID;
  sdp_settings st;
  sdp_default_settings(&st);
  if (settings) st = *settings;
  if (!settings_ok(&st)) return SDP_E_INVALID;
  sdp_ctx* c = new sdp_ctx();
  c->st = st;
  c->stream = (cudaStream_t)stream;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) {
    delete c;
    set_err(cudaGetErrorString(e), __FILE__, __LINE__);
    return SDP_E_CUDA;
  }
  *out = c;
  return SDP_OK;
}

static void free_group_cache(sdp_ctx* c);

extern "C" void sdp_destroy(sdp_ctx* c) {
  if (!c) return;
  free_group_cache(c);
  for (auto& kv : c->projs) sdp_destroy(kv.second);
  c->projs.clear();
  ctx_free(c);
  delete c;
}

extern "C" int sdp_update_settings(sdp_ctx* c, const sdp_settings* s) {
  if (!c || !s || !settings_ok(s)) return SDP_E_INVALID;
  int mf_changed = (s->mode_frac != c->st.mode_frac) || (s->expand_frac != c->st.expand_frac);
  if (c->ready && mf_changed) return SDP_E_STATE;
  c->st = *s;
  c->inst.rho = s->rho;
  c->inst.sigma = s->sigma;
  c->inst.alpha = s->alpha;
  c->inst.prec = s->precision;
  return SDP_OK;
}

// Build sparse operators and factor K on the host, upload everything.
extern "C" int sdp_setup(sdp_ctx* c, int n, const double* C, int mc, long nnz, const int* cp, const int* ci,
                         const int* cj, const double* cv, const double* b, int on_device) {
  if (!c || n < 1 || mc < 0 || nnz < 0 || !C || (mc > 0 && (!b || (nnz > 0 && (!cp || !ci || !cj || !cv)))))
    return SDP_E_INVALID;
  std::vector<int> hp(nnz), hi(nnz), hj(nnz);
  std::vector<double> hv(nnz), hb(mc), hC((size_t)n * n);
  if (on_device) {
    if (nnz) {
      CK(cudaMemcpy(hp.data(), cp, sizeof(int) * nnz, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(hi.data(), ci, sizeof(int) * nnz, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(hj.data(), cj, sizeof(int) * nnz, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(hv.data(), cv, sizeof(double) * nnz, cudaMemcpyDeviceToHost));
    }
    if (mc) CK(cudaMemcpy(hb.data(), b, sizeof(double) * mc, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(hC.data(), C, sizeof(double) * (size_t)n * n, cudaMemcpyDeviceToHost));
  } else {
    if (nnz) {
      memcpy(hp.data(), cp, sizeof(int) * nnz);
      memcpy(hi.data(), ci, sizeof(int) * nnz);
      memcpy(hj.data(), cj, sizeof(int) * nnz);
      memcpy(hv.data(), cv, sizeof(double) * nnz);
    }
    if (mc) memcpy(hb.data(), b, sizeof(double) * mc);
    memcpy(hC.data(), C, sizeof(double) * (size_t)n * n);
  }
  for (long t = 0; t < nnz; ++t)
    if (hp[t] < 0 || hp[t] >= mc || hi[t] < 0 || hj[t] >= n || hi[t] > hj[t]) return SDP_E_INVALID;
  for (size_t q = 0; q < hC.size(); ++q)
    if (!std::isfinite(hC[q])) return SDP_E_NUMERICAL;
  for (int p = 0; p < mc; ++p)
    if (!std::isfinite(hb[p])) return SDP_E_NUMERICAL;
  for (long t = 0; t < nnz; ++t)
    if (!std::isfinite(hv[t])) return SDP_E_NUMERICAL;
  HostSetup H;
  int rc = host_setup(n, mc, nnz, hp.data(), hi.data(), hj.data(), hv.data(), c->st.sigma, c->st.rho, &H);
  if (rc) return rc;
  ctx_free(c);
  c->L = make_layout(n, mc, nnz, H.nent, H.nF, c->st);
  c->dbytes = layout_bytes(c->L, nullptr, nullptr);
  cudaError_t e = cudaMalloc(&c->dmem, c->dbytes);
  if (e != cudaSuccess) {
    c->dmem = nullptr;
    set_err(cudaGetErrorString(e), __FILE__, __LINE__);
    return SDP_E_NOMEM;
  }
  layout_bytes(c->L, &c->inst, c->dmem);
  Inst& I = c->inst;
  I.rho = c->st.rho;
  I.sigma = c->st.sigma;
  I.alpha = c->st.alpha;
  I.prec = c->st.precision;
  // K part
  size_t nk = H.k_col.size();
  c->kbytes = (nk * (sizeof(int) + sizeof(double)) + (size_t)H.nF * H.nF * sizeof(double) + 3 * 256);
  e = cudaMalloc(&c->dK, c->kbytes);
  if (e != cudaSuccess) {
    ctx_free(c);
    set_err(cudaGetErrorString(e), __FILE__, __LINE__);
    return SDP_E_NOMEM;
  }
  size_t o1 = (nk * sizeof(int) + 255) / 256 * 256;
  size_t o2 = o1 + (nk * sizeof(double) + 255) / 256 * 256;
  I.k_col = (int*)c->dK;
  I.k_val = (double*)(c->dK + o1);
  I.Lf = (double*)(c->dK + o2);
  cudaStream_t s = c->stream;
  CK(cudaMemsetAsync(c->dmem, 0, c->dbytes, s));
  // C into padded layout
  std::vector<double> pad((size_t)I.ld * n, 0.0);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) pad[(size_t)i + (size_t)j * I.ld] = 0.5 * (hC[i + (size_t)j * n] + hC[j + (size_t)i * n]);
  CK(cudaMemcpyAsync(I.C, pad.data(), sizeof(double) * pad.size(), cudaMemcpyHostToDevice, s));
  if (mc) CK(cudaMemcpyAsync(I.b, hb.data(), sizeof(double) * mc, cudaMemcpyHostToDevice, s));
  if (H.nent) {
    CK(cudaMemcpyAsync(I.ent_i, H.ent_i.data(), sizeof(int) * H.nent, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(I.ent_j, H.ent_j.data(), sizeof(int) * H.nent, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(I.ent_ptr, H.ent_ptr.data(), sizeof(int) * (H.nent + 1), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(I.ent_con, H.ent_con.data(), sizeof(int) * H.ent_con.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(I.ent_val, H.ent_val.data(), sizeof(double) * H.ent_val.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(I.con_ent, H.con_ent.data(), sizeof(int) * H.con_ent.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(I.con_w, H.con_w.data(), sizeof(double) * H.con_w.size(), cudaMemcpyHostToDevice, s));
  }
  if (mc) {
    CK(cudaMemcpyAsync(I.con_ptr, H.con_ptr.data(), sizeof(int) * (mc + 1), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(I.kdiag, H.kdiag.data(), sizeof(double) * mc, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(I.isD, H.isD.data(), sizeof(int) * mc, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(I.fpos, H.fpos.data(), sizeof(int) * mc, cudaMemcpyHostToDevice, s));
    if (H.nF) CK(cudaMemcpyAsync(I.Flist, H.Flist.data(), sizeof(int) * H.nF, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(I.k_ptr, H.k_ptr.data(), sizeof(int) * (mc + 1), cudaMemcpyHostToDevice, s));
    if (nk) {
      CK(cudaMemcpyAsync(I.k_col, H.k_col.data(), sizeof(int) * nk, cudaMemcpyHostToDevice, s));
      CK(cudaMemcpyAsync(I.k_val, H.k_val.data(), sizeof(double) * nk, cudaMemcpyHostToDevice, s));
    }
    if (H.nF)
      CK(cudaMemcpyAsync(I.Lf, H.Lf.data(), sizeof(double) * H.Lf.size(), cudaMemcpyHostToDevice, s));
  }
  // sparse-position mask
  std::vector<uint32_t> mask(((size_t)I.ld * n + 31) / 32, 0u);
  for (int e2 = 0; e2 < H.nent; ++e2) {
    size_t q = (size_t)H.ent_i[e2] + (size_t)H.ent_j[e2] * I.ld;
    size_t qt = (size_t)H.ent_j[e2] + (size_t)H.ent_i[e2] * I.ld;
    mask[q >> 5] |= 1u << (q & 31);
    mask[qt >> 5] |= 1u << (qt & 31);
  }
  CK(cudaMemcpyAsync(I.smask, mask.data(), sizeof(uint32_t) * mask.size(), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  c->ready = true;
  c->status = SDP_OK;
  c->cert_kind = 0;
  c->k = 0;
  return SDP_OK;
}

extern "C" unsigned long long sdp_footprint_bytes(int n, int m, long nnz, int precision) {
  sdp_settings st;
  sdp_default_settings(&st);
  st.precision = precision;
  Layout L = make_layout(n, m, nnz, (int)std::min<long>(nnz, (long)n * (n + 1) / 2), 1, st);
  return (unsigned long long)layout_bytes(L, nullptr, nullptr) + (unsigned long long)nnz * 12ull;
}

// ---------------------------------------------------------------------------
// Group engine
// ---------------------------------------------------------------------------
#include "engine.inc"
