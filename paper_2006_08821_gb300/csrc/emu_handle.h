// The solver handle behind the C ABI of include/emu.h: device buffers, launch
// shapes, profiling state and the parameters of one mesh. Shared by the host
// translation units (setup and Newton loop, bones and joints).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "emu_bones.h"
#include "emu_bones_host.h"
#include "emu_internal.h"
#include "emu_kernels.cuh"
#include "emu_mixed.cuh"
#include "emu_pcg.h"
#include "emu_syrk05.h"

namespace emu {
// Cyclic Jacobi eigen-decomposition of a symmetric N x N matrix (row-major):
// A is overwritten (its diagonal holds the eigenvalues), V receives the
// eigenvectors as columns.
void host_jacobi_eig(std::vector<double>& A, std::vector<double>& V, int N);

struct DevBuf {
  void* p;
  size_t bytes;
};
}  // namespace emu

// emu_handle is a global type (declared in emu.h); its members use the
// library's own types.
using namespace emu;

struct emu_handle {
  emu_params prm;
  emu_allocator alloc;
  bool has_alloc = false;
  cudaStream_t st = nullptr;
  int device = 0;  // the CUDA device current at emu_create (all memory lives there)
  int64_t n = 0, m = 0;
  int sms = 0;
  int kmodes = 16;
  bool mixed = false;
  bool escalated = false;  // a mixed handle running the FP64 kernels for the rest of a solve
  bool fform = false;      // the F-form of Sec. 3.2.1 (FP64): R holds F, Uw the 9 x 9 factors
  std::vector<emu::DevBuf> bufs;

  double mu_ref = 0, alpha = 0, kappa = 0;
  double gref = 0;  // ||g(I)||
  bool gref_valid = false;
  double floor = 0;  // 1e-12 sqrt(sum (V mu)^2)
  std::vector<double> V_h;

  // device arrays
  int4* tet = nullptr;
  double *Dinv = nullptr, *V = nullptr, *c = nullptr, *w = nullptr, *mu = nullptr, *lam = nullptr, *u = nullptr,
         *ka = nullptr;
  double* gam64 = nullptr;
  float* gam32 = nullptr;
  double *R = nullptr, *s = nullptr, *q = nullptr, *dq = nullptr, *q0 = nullptr, *g = nullptr;
  double *y64 = nullptr, *d64 = nullptr, *Uw64 = nullptr;
  float *y32 = nullptr, *d32 = nullptr, *Uw32 = nullptr;
  double* contrib = nullptr;
  float* contrib32 = nullptr;  // mixed: FP32 corner terms of the direction
  double* b = nullptr;
  double *pr = nullptr, *pu = nullptr, *pw = nullptr, *pp = nullptr, *ps = nullptr;
  // mixed path: FP32 constants and state, FP32 CG work vectors
  float *Dinv32 = nullptr, *V32 = nullptr, *c32 = nullptr, *w32 = nullptr, *mu32 = nullptr, *lam32 = nullptr,
        *u32 = nullptr, *ka32 = nullptr, *E32 = nullptr, *g32 = nullptr, *dq32 = nullptr, *b32 = nullptr,
        *r32 = nullptr, *e32 = nullptr;
  float4* quat = nullptr;
  float *uh32 = nullptr, *ul32 = nullptr;  // q - Q as a float pair (hi, lo), 3n each
  float* E0 = nullptr;     // 9m: G_i Q - I of the FP32 D_m^-1
  double* Qrest = nullptr;  // 3n rest positions
  float *val32 = nullptr, *ldinv32 = nullptr;
  float *fr = nullptr, *fu = nullptr, *fw = nullptr, *fp = nullptr, *fs = nullptr;
  // coarse space of the ACAP preconditioner: the low-rank basis Phi (n x 16)
  // and the pseudo-inverse of Phi^T L Phi
  double* phi64 = nullptr;
  float* phi32 = nullptr;
  double* Einv = nullptr;
  double* lam_add = nullptr;  // F-form: Phi^T K Phi (48 x 48) and 48 zeros, the capacitance's addend
  bool coarse_ready = false;
  // register-resident FP32 CG: exchange buffer, partial sums, launch shape
  float4* ug32 = nullptr;                // 2 n exchange entries of the FP32 CG
  unsigned* sync32 = nullptr;             // its barrier words
  float* part32 = nullptr;
  float* aphi32 = nullptr;                // rows of L Phi for the pipelined FP32 CG
  bool aphi_ready = false;
  bool syrk05 = false;  // capacitance on the tcgen05 kernel (else mma.sync)
  // constant external force (Sec. 3.4): generalized force nu = W G K^-1 f
  bool has_force = false;
  double* nu64 = nullptr;  // 9m (allocated on first use)
  float* nu32 = nullptr;   // 9m, mixed path
  Syrk05Maps syrk05_maps;  // its tensor maps of Uw32, gam32, y32, sw32
  float* sw32 = nullptr;    // sqrt of the ACAP weights (m)
  int grid32 = 0, rpt32 = 0;
  // the partitioned system of the pipelined FP32 CG (emu_cgpart.h)
  bool cg_part = false;  // built at creation (mixed path, pipelined shape)
  int32_t *cg_perm = nullptr, *cg_off = nullptr, *cg_rowptr = nullptr, *cg_col = nullptr;
  float *cg_val = nullptr, *cg_dinv = nullptr, *cg_phi = nullptr, *cg_aphi = nullptr;
  uint32_t* cg_loc = nullptr;
  int cg_lw = 0, cg_degree = 1;
  float cg_c0 = 1.f, cg_c1[kChebMax] = {0}, cg_c2[kChebMax] = {0};
  double cg_lmax = 0.0;            // Gershgorin bound of the local blocks (the polynomial's interval)
  int cg64_rows = 128;             // rows per block of the FP64 CG (grid_pcg3 = ceil(n / cg64_rows), capped)
  bool tuned = false;              // set-up ran the autotuner (emu_params.autotune)
  double q_tol = 1e-8;
  double dq_tol_now = 5e-2;  // dq tolerance of the current solve call
  double dq_tol_base = 0.0;  // tighter dq tolerance a stalled solve settled on (0: params.dq_tol)
  double sigma0_now = 1.0;   // first line-search trial: params.ls_sigma0, or 1 after a stall
  double *part_grad = nullptr, *part_dir = nullptr, *part_ls = nullptr, *part_pcg = nullptr, *cpart = nullptr;
  double* z = nullptr;
  double* cfull = nullptr;  // summed capacitance entries
  double* scratch16 = nullptr;  // n x 16 mode vectors
  double* small = nullptr;      // 256 doubles of small-matrix exchange
  DevScalars* sc = nullptr;
  DevScalars* sc_host = nullptr;  // pinned
  double* o6_host = nullptr;       // pinned: residual sums of the refresh rounds (16)
  cudaEvent_t wait_ev = nullptr;   // marks the work a solve task waits for
  // one Newton iteration (direction .. update, next gradient) as a CUDA graph
  cudaGraphExec_t iter_exec = nullptr;
  double iter_exec_dq = -1.0;      // dq tolerance the graph was captured with
  double iter_exec_sigma0 = -1.0;  // and first trial step
  bool graphs_ok = true;           // false once a capture failed (direct launches)
  int64_t iter_graph_kernels = 0;  // kernel launches in one graph launch
  GridBarrier* bar = nullptr;
  // Laplacian and pins
  int32_t *rowptr = nullptr, *col = nullptr;
  double *val = nullptr, *ldinv = nullptr, *bfix = nullptr, *qfix = nullptr;
  uint8_t* is_fixed = nullptr;
  int32_t *slot_ptr = nullptr, *slot_idx = nullptr;
  // ---- affine bones and joints (Sec. 3.3; see emu_bones.h) ----
  bool has_bones = false;   // some tet belongs to a bone
  int nb = 0;               // bones (pinned and free)
  int nfb = 0;              // free bones: Newton variables of their own
  int npts = 0;             // joint points (rows of J)
  int njv = 0;              // vertices with a J entry
  double eps_bone = -1e-3, eps_joint = -1e-4;
  double Vbar = 0.0;        // mean rest volume
  double kj = 0.0;          // final joint penalty Vbar^(1/3) / |eps_joint|
  // host copies
  std::vector<int32_t> tkind_h, btets_h, bptr_h, rep_h, bvert_h, bvptr_h;
  std::vector<std::vector<int32_t>> bverts_h;   // vertices of every bone
  std::vector<int> free_index_h;                // bone -> free-bone index, -1 if pinned
  std::vector<double> Vb_h, wb_h, mub_h, lamb_h;
  std::vector<double> w_h;                      // ACAP weights per tet (with the bone penalty)
  std::vector<int32_t> jv_h;
  std::vector<double> jw_h, JJinv_h, sgn_h;     // sgn: npts x kMaxFreeBones, (J zeta_b)_r
  std::vector<uint8_t> jfree_h;
  std::vector<int32_t> frowptr_h, fcol_h;       // final-solve Laplacian (CSR)
  std::vector<double> fval_h, fldinv_h, zrhs_h;
  std::vector<uint8_t> fin_fixed_h;
  double Ainv_h[kMaxFreeBones * kMaxFreeBones] = {0};
  // device arrays
  int32_t *tkind = nullptr, *btets = nullptr, *bvert = nullptr;
  double *gbar = nullptr, *cconst = nullptr, *bpart = nullptr, *cadd = nullptr, *bst = nullptr, *Qd = nullptr;
  int32_t* jv = nullptr;
  double *jw = nullptr, *Sinv = nullptr, *JJinv = nullptr, *Y64 = nullptr, *jlam = nullptr;
  float* Y32 = nullptr;
  uint8_t *jfree = nullptr, *jmask = nullptr;
  int32_t *frowptr = nullptr, *fcol = nullptr;
  double *fval = nullptr, *fldinv = nullptr, *zeta = nullptr, *fdt = nullptr;
  double *phi_fin = nullptr, *Einv_fin = nullptr;  // coarse space of the final solve's CG
  uint8_t* fin_fixed = nullptr;
  int64_t fnnz = 0;
  BoneArgs bargs() const;
  JointArgs jargs() const;
  FinalArgs fargs() const;

  // launch shapes
  int grid_tet = 1, grid_syrk = 1, grid_pcg3 = 1, grid_pcg16 = 1;
  int grid_tet4 = 1;  // one wave of the 4-blocks-per-SM mixed gradient and line-search kernels

  // profiling: event pairs per phase, resolved at the next host sync
  struct Pending {
    int phase;
    int launches;
    cudaEvent_t e0, e1;
  };
  bool prof_on = false;
  double prof_ms[EMU_N_PHASES] = {0};
  int32_t prof_cnt[EMU_N_PHASES] = {0};
  int64_t launches = 0;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<Pending> pending;
  cudaEvent_t cur_e0 = nullptr;

  cudaEvent_t ev_get() {
    if (!ev_pool.empty()) {
      cudaEvent_t e = ev_pool.back();
      ev_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void ph_begin() {
    if (!prof_on) return;
    cur_e0 = ev_get();
    cudaEventRecord(cur_e0, st);
  }
  void ph_end(int phase, int nlaunch) {
    launches += nlaunch;
    if (!prof_on) return;
    cudaEvent_t e1 = ev_get();
    cudaEventRecord(e1, st);
    pending.push_back({phase, nlaunch, cur_e0, e1});
  }
  // call after the stream was synchronised
  void prof_flush() {
    for (auto& p_ : pending) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, p_.e0, p_.e1);
      prof_ms[p_.phase] += ms;
      prof_cnt[p_.phase] += p_.launches;
      ev_pool.push_back(p_.e0);
      ev_pool.push_back(p_.e1);
    }
    pending.clear();
  }
  void prof_destroy() {
    prof_flush();
    for (auto e : ev_pool) cudaEventDestroy(e);
    ev_pool.clear();
  }

  bool dry = false;       // count bytes only (memory estimate)
  size_t dry_bytes = 0;
  void* dalloc(size_t bytes) {
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~size_t(255);
    if (dry) {
      dry_bytes += bytes;
      return reinterpret_cast<void*>(uintptr_t(256));
    }
    void* p = nullptr;
    if (has_alloc) {
      p = alloc.alloc(alloc.ctx, bytes, (void*)st);
    } else {
      if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
    }
    if (p) bufs.push_back({p, bytes});
    return p;
  }
  template <typename T> bool get(T*& out, size_t count) {
    out = static_cast<T*>(dalloc(count * sizeof(T)));
    return out != nullptr;
  }
  void release() {
    if (st) cudaStreamSynchronize(st);
    prof_destroy();
    for (auto& b_ : bufs) {
      if (has_alloc)
        alloc.free(alloc.ctx, b_.p, b_.bytes, (void*)st);
      else
        cudaFree(b_.p);
    }
    bufs.clear();
    if (sc_host) cudaFreeHost(sc_host);
    sc_host = nullptr;
    if (o6_host) cudaFreeHost(o6_host);
    o6_host = nullptr;
    if (wait_ev) cudaEventDestroy(wait_ev);
    wait_ev = nullptr;
    if (iter_exec) cudaGraphExecDestroy(iter_exec);
    iter_exec = nullptr;
  }

  template <typename TW> TetArgs<TW> args();

  PcgArgsT<double> pcg64(const double* rhs, double* x, double tol) {
    PcgArgsT<double> a;
    a.n = n;
    a.rowptr = rowptr;
    a.col = col;
    a.val = val;
    a.dinv = ldinv;
    a.b = rhs;
    a.x = x;
    a.r = pr;
    a.u = pu;
    a.w = pw;
    a.p = pp;
    a.s = ps;
    a.partials = part_pcg;
    a.bar = bar;
    a.tol = tol;
    a.max_iter = prm.pcg_max;
    a.iters_out = &sc->pcg_iters;
    a.fail_out = &sc->pcg_fail;
    a.timeout_out = &sc->barrier_timeout;
    a.last_iters = nullptr;
    a.relres_out = nullptr;
    a.phi = coarse_ready ? phi64 : nullptr;
    a.Einv = coarse_ready ? Einv : nullptr;
    return a;
  }
  PcgArgsT<float> pcg32(const float* rhs, float* x, double tol) {
    PcgArgsT<float> a;
    a.n = n;
    a.rowptr = rowptr;
    a.col = col;
    a.val = val32;
    a.dinv = ldinv32;
    a.b = rhs;
    a.x = x;
    a.r = fr;
    a.u = fu;
    a.w = fw;
    a.p = fp;
    a.s = fs;
    a.partials = part_pcg;
    a.bar = bar;
    a.tol = tol;
    a.max_iter = prm.pcg_max;
    a.iters_out = &sc->pcg_iters;
    a.fail_out = &sc->pcg_fail;
    a.timeout_out = &sc->barrier_timeout;
    a.last_iters = nullptr;
    a.relres_out = nullptr;
    a.phi = coarse_ready ? phi32 : nullptr;
    a.Einv = coarse_ready ? Einv : nullptr;
    return a;
  }
  MixArgs margs() {
    MixArgs a;
    a.m = m;
    a.n = n;
    a.tet = tet;
    a.Dinv = Dinv32;
    a.V = V32;
    a.c = c32;
    a.w = w32;
    a.sw = sw32;
    a.mu = mu32;
    a.lam = lam32;
    a.ka = ka32;
    a.u = u32;
    a.gam = gam32;
    a.quat = quat;
    a.E = E32;
    a.q = q;
    a.Q = Qrest;
    a.uh = uh32;
    a.ul = ul32;
    a.E0 = E0;
    a.dq = dq32;
    a.g = g32;
    a.y = y32;
    a.d = d32;
    a.Uw = Uw32;
    a.contrib = contrib;
    a.contrib32 = contrib32;
    a.b32 = b32;
    a.z = z;
    a.sc = sc;
    a.partials = part_grad;
    a.tkind = tkind;
    a.bone_st = bst;
    a.nu = has_force ? nu32 : nullptr;
    return a;
  }
};

template <> inline TetArgs<double> emu_handle::args<double>() {
  TetArgs<double> a;
  a.m = m;
  a.n = n;
  a.tet = tet;
  a.Dinv = Dinv;
  a.V = V;
  a.c = c;
  a.w = w;
  a.mu = mu;
  a.lam = lam;
  a.u = u;
  a.ka = ka;
  a.gam = gam64;
  a.R = R;
  a.s = s;
  a.q = q;
  a.dq = dq;
  a.g = g;
  a.y = y64;
  a.d = d64;
  a.Uw = Uw64;
  a.contrib = contrib;
  a.z = z;
  a.sc = sc;
  a.partials = part_grad;
  a.tkind = tkind;
  a.bone_st = bst;
  a.nu = has_force ? nu64 : nullptr;
  return a;
}
template <> inline TetArgs<float> emu_handle::args<float>() {
  TetArgs<float> a;
  a.m = m;
  a.n = n;
  a.tet = tet;
  a.Dinv = Dinv;
  a.V = V;
  a.c = c;
  a.w = w;
  a.mu = mu;
  a.lam = lam;
  a.u = u;
  a.ka = ka;
  a.gam = gam32;
  a.R = R;
  a.s = s;
  a.q = q;
  a.dq = dq;
  a.g = g;
  a.y = y32;
  a.d = d32;
  a.Uw = Uw32;
  a.contrib = contrib;
  a.z = z;
  a.sc = sc;
  a.partials = part_grad;
  a.tkind = tkind;
  a.bone_st = bst;
  a.nu = has_force ? nu64 : nullptr;
  return a;
}

