// C-ABI of the batched ABD-IPC step: workspace layout, state I/O, the Newton
// driver (host orchestration of the device kernels) and diagnostics.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/ipc_b300.h"
#include "ctx.h"
#include "kernels.h"

using namespace ipc;

namespace {

#define CK(call)                                                                 \
  do {                                                                           \
    cudaError_t _e = (call);                                                     \
    if (_e != cudaSuccess) {                                                     \
      if (ctx) ctx->err = std::string(#call) + ": " + cudaGetErrorString(_e);    \
      return IPC_ECUDA;                                                          \
    }                                                                            \
  } while (0)

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

// ---- per-kernel-class launch counts and event timing
enum Kc {
  KC_PREDICT, KC_CVPOS, KC_OBJBOX, KC_BROAD, KC_BARRIER, KC_TET, KC_BODY, KC_ASSEMBLE, KC_GRAD, KC_PRECOND,
  KC_PCGINIT, KC_PAIRSPMV, KC_FRICSPMV, KC_SPMV, KC_PCGUPD, KC_NEWTON, KC_ACCD, KC_ENERGY, KC_LS, KC_MISC,
  KC_PCGITER, KC_COUNT
};
const char* KC_NAME[KC_COUNT] = {"predict",      "cv_pos",      "obj_box",     "broad_phase", "barrier",
                                 "tet_elastic",  "body_abd",    "assemble",    "gradient",    "precond",
                                 "pcg_init",     "pair_matvec", "fric_matvec", "pcg_matvec",  "pcg_update",
                                 "newton_check", "accd",        "ls_energy",   "ls_update",   "misc",
                                 "pcg_iter"};

cudaEvent_t take_ev(ipc_ctx* ctx) {
  if (!ctx->ev_free.empty()) {
    cudaEvent_t e = ctx->ev_free.back();
    ctx->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

// launches on stream `st` (the ctx stream unless a side stream is named),
// timed per class when profiling is on
template <class F>
void KL(ipc_ctx* ctx, int kind, F&& f, cudaStream_t st = nullptr) {
  if (!ctx->prof_on) {
    ctx->launches += f();
    return;
  }
  if (!st) st = ctx->stream;
  cudaEvent_t a = take_ev(ctx), b = take_ev(ctx);
  cudaEventRecord(a, st);
  int n = f();
  cudaEventRecord(b, st);
  ctx->launches += n;
  ctx->prof_launches[kind] += n;
  ctx->pending.push_back({kind, a, b});
}

// the first n side streams start after everything issued so far on the
// main stream s (the ctx stream, or the stream capturing a graph body) ...
int side_set(const ipc_ctx* ctx, cudaStream_t s) {
  for (int i = 0; i < 3; ++i)
    if (s == ctx->cap[i]) return 1 + i;
  return 0;
}
// side stream i of main stream s
cudaStream_t side_of(const ipc_ctx* ctx, cudaStream_t s, int i) { return ctx->side[side_set(ctx, s)][i]; }
void fork_side(ipc_ctx* ctx, cudaStream_t s, int n = 2) {
  const int k = side_set(ctx, s);
  cudaEventRecord(ctx->ev_fork[k], s);
  for (int i = 0; i < n; ++i) cudaStreamWaitEvent(ctx->side[k][i], ctx->ev_fork[k], 0);
}
// ... and s continues only after them
void join_side(ipc_ctx* ctx, cudaStream_t s, int n = 2) {
  const int k = side_set(ctx, s);
  for (int i = 0; i < n; ++i) {
    cudaEventRecord(ctx->ev_join[k][i], ctx->side[k][i]);
    cudaStreamWaitEvent(s, ctx->ev_join[k][i], 0);
  }
}

// resolve recorded event pairs (the stream has been synchronised)
void prof_flush(ipc_ctx* ctx) {
  for (auto& pe : ctx->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pe.a, pe.b) == cudaSuccess) ctx->prof_ms[pe.kind] += ms;
    ctx->ev_free.push_back(pe.a);
    ctx->ev_free.push_back(pe.b);
  }
  ctx->pending.clear();
}

// Walks every device array in a fixed order; with ws == nullptr only sums
// sizes.  Static tables are copied from the pack when `upload` is set.
struct Carver {
  char* base;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += align256(std::max<size_t>(count, 1) * sizeof(T));
    return p;
  }
};

template <class T>
const T* carve_copy(Carver& cv, const std::vector<T>& v, std::vector<std::pair<const void*, std::pair<void*, size_t>>>& up) {
  T* p = cv.take<T>(v.size());
  if (p && !v.empty()) up.push_back({v.data(), {p, v.size() * sizeof(T)}});
  return p;
}

struct Extra {
  std::vector<int> env_pair_off_i, has_driven;
};

void carve(const Pack& pk, const ipc_params& prm, Carver& c, Dev& d, Extra& ex,
           std::vector<std::pair<const void*, std::pair<void*, size_t>>>& up) {
  d.n_envs = pk.n_envs;
  d.n_rows = pk.n_rows;
  d.n_tets = pk.n_tets;
  d.n_cv = pk.n_cv;
  d.n_tri = pk.n_tri;
  d.n_edge = pk.n_edge;
  d.n_obj = pk.n_obj;
  d.n_bodies = pk.n_bodies;
  d.n_chunks = pk.n_chunks;
  d.n_coated = pk.n_coated;
  d.n_blocks = pk.n_sell_blocks;
  d.n_pairs_cap = pk.n_pairs_cap;
  d.h = prm.dt;
  for (int k = 0; k < 3; ++k) d.grav[k] = prm.gravity[k];
  d.dhat = prm.dhat;
  d.kappa = prm.kappa;
  d.newton_tol = prm.newton_tol;
  d.pcg_tol = prm.pcg_rel_tol;
  d.accd_s = prm.accd_s;
  d.al_kappa = prm.al_kappa;
  d.ee_moll = prm.ee_mollifier;
  d.fr_mu = prm.friction_mu;
  d.fr_eh = prm.friction_eps_v * prm.dt;
  d.spmv_unroll = 0;
  d.pcg_fused = prm.pcg_fused;
  d.pcg_grid = 148;
  d.pcg_grid_fused = 148;
  d.pcg_iter_bound = 1;
  d.pcg_multi = prm.pcg_iters_per_launch;
  d.pcg_grid_multi = 148;
  d.asm_block = 128;
  d.pairs_grid = 148 * 8;
  d.newton_max = prm.newton_max;
  d.pcg_max = prm.pcg_max;
  d.ls_max = prm.ls_max;
  d.accd_max = prm.accd_max;
  d.al_max = prm.al_max;
  d.abs_after = prm.newton_abs_after;
  d.prec = prm.precision ? 1 : 0;

  ex.env_pair_off_i.assign(pk.env_pair_off.begin(), pk.env_pair_off.end());
  ex.has_driven.assign(pk.n_envs, 0);
  for (int e = 0; e < pk.n_envs; ++e)
    for (int r = pk.env_row_off[e]; r < pk.env_row_off[e + 1]; ++r)
      if (pk.row_kind[r] == ROW_ATTACHED || pk.row_kind[r] == ROW_BODY_DRIVEN) { ex.has_driven[e] = 1; break; }

  d.env_row_off = carve_copy(c, pk.env_row_off, up);
  d.env_tet_off = carve_copy(c, pk.env_tet_off, up);
  d.env_cv_off = carve_copy(c, pk.env_cv_off, up);
  d.env_tri_off = carve_copy(c, pk.env_tri_off, up);
  d.env_edge_off = carve_copy(c, pk.env_edge_off, up);
  d.env_obj_off = carve_copy(c, pk.env_obj_off, up);
  d.env_body_off = carve_copy(c, pk.env_body_off, up);
  d.env_chunk_off = carve_copy(c, pk.env_chunk_off, up);
  d.env_coated_off = carve_copy(c, pk.env_coated_off, up);
  d.env_pair_cap = carve_copy(c, pk.env_pair_cap, up);
  d.env_pair_off = carve_copy(c, ex.env_pair_off_i, up);
  d.env_has_driven = carve_copy(c, ex.has_driven, up);
  d.env_mu = carve_copy(c, pk.env_mu, up);
  d.env_lam = carve_copy(c, pk.env_lam, up);
  d.cta_env = carve_copy(c, pk.cta_env, up);
  d.row_mass = carve_copy(c, pk.row_mass, up);
  d.row_kind = carve_copy(c, pk.row_kind, up);
  d.row_body = carve_copy(c, pk.row_body, up);
  d.row_xbar = carve_copy(c, pk.row_xbar, up);
  d.vt_ptr = carve_copy(c, pk.vt_ptr, up);
  d.vt_src = carve_copy(c, pk.vt_src, up);
  d.tets = carve_copy(c, pk.tets, up);
  d.Dm_inv = carve_copy(c, pk.Dm_inv, up);
  d.tet_vol = carve_copy(c, pk.tet_vol, up);
  d.chunk_slots = carve_copy(c, pk.chunk_slots, up);
  d.chunk_ptr = carve_copy(c, pk.chunk_ptr, up);
  d.sell_col = carve_copy(c, pk.sell_col, up);
  d.asm_ptr = carve_copy(c, pk.asm_ptr, up);
  d.asm_src = carve_copy(c, pk.asm_src, up);
  d.body_row = carve_copy(c, pk.body_row, up);
  d.body_env = carve_copy(c, pk.body_env, up);
  d.body_cv_begin = carve_copy(c, pk.body_cv_begin, up);
  d.body_nv = carve_copy(c, pk.body_nv, up);
  d.body_mass = carve_copy(c, pk.body_mass, up);
  d.body_S = carve_copy(c, pk.body_S, up);
  d.body_vol = carve_copy(c, pk.body_vol, up);
  d.body_kappa = carve_copy(c, pk.body_kappa, up);
  d.body_driven = carve_copy(c, pk.body_driven, up);
  d.cv_row = carve_copy(c, pk.cv_row, up);
  d.cv_body = carve_copy(c, pk.cv_body, up);
  d.cv_obj = carve_copy(c, pk.cv_obj, up);
  d.cv_uid = carve_copy(c, pk.cv_uid, up);
  d.cv_xbar = carve_copy(c, pk.cv_xbar, up);
  d.cv_area = carve_copy(c, pk.cv_area, up);
  d.cv_fixed = carve_copy(c, pk.cv_fixed, up);
  d.tri = carve_copy(c, pk.tri, up);
  d.tri_obj = carve_copy(c, pk.tri_obj, up);
  d.edge = carve_copy(c, pk.edge, up);
  d.edge_obj = carve_copy(c, pk.edge_obj, up);
  d.edge_area = carve_copy(c, pk.edge_area, up);
  d.edge_len2 = carve_copy(c, pk.edge_len2, up);
  d.obj_env = carve_copy(c, pk.obj_env, up);
  d.obj_local = carve_copy(c, pk.obj_local, up);
  d.obj_cv_begin = carve_copy(c, pk.obj_cv_begin, up);
  d.obj_cv_end = carve_copy(c, pk.obj_cv_end, up);
  d.obj_tri_begin = carve_copy(c, pk.obj_tri_begin, up);
  d.obj_tri_end = carve_copy(c, pk.obj_tri_end, up);
  d.obj_edge_begin = carve_copy(c, pk.obj_edge_begin, up);
  d.obj_edge_end = carve_copy(c, pk.obj_edge_end, up);
  d.obj_size = carve_copy(c, pk.obj_size, up);
  d.obj_exclude = carve_copy(c, pk.obj_exclude, up);
  d.coated_row = carve_copy(c, pk.coated_row, up);
  for (int k = 0; k < 3; ++k) {
    d.bv_perm[k] = carve_copy(c, pk.bv_perm[k], up);
    d.bv_cl_obj[k] = carve_copy(c, pk.bv_cl_obj[k], up);
    d.bv_sc_obj[k] = carve_copy(c, pk.bv_sc_obj[k], up);
    d.obj_cl_begin[k] = carve_copy(c, pk.obj_cl_begin[k], up);
    d.obj_sc_begin[k] = carve_copy(c, pk.obj_sc_begin[k], up);
    d.bv_n_cl[k] = (int)pk.bv_cl_obj[k].size();
    d.bv_n_sc[k] = (int)pk.bv_sc_obj[k].size();
  }
  // dynamic
  size_t R3 = 3 * (size_t)pk.n_rows;
  d.x = c.take<double>(R3);
  d.v = c.take<double>(R3);
  d.xn = c.take<double>(R3);
  d.xt = c.take<double>(R3);
  d.s_tgt = c.take<double>(R3);
  d.lam = c.take<double>(R3);
  d.p = c.take<double>(R3);
  d.g = c.take<double>(R3);
  d.r = c.take<double>(R3);
  d.z = c.take<double>(R3);
  d.d = c.take<double>(R3);
  d.db = c.take<double>(R3);
  d.z4 = c.take<float4>((size_t)pk.n_rows);
  d.d4 = c.take<float4>((size_t)pk.n_rows);
  d.d4b = c.take<float4>((size_t)pk.n_rows);
  d.q4 = c.take<float4>((size_t)pk.n_rows);
  d.row_touch = c.take<uint8_t>((size_t)pk.n_rows);
  d.pcg_list = c.take<int>((size_t)pk.n_envs);
  d.pcg_pair_off = c.take<int>((size_t)pk.n_envs + 1);
  d.pcg_row_off = c.take<int>((size_t)pk.n_envs + 1);
  d.pcg_item = c.take<int2>((size_t)pk.n_rows / 128);
  d.pcg_pitem = c.take<int2>((size_t)pk.n_pairs_cap / 8 + (size_t)pk.n_envs);
  d.pcg_fitem = c.take<int2>((size_t)pk.n_pairs_cap / 128 + (size_t)pk.n_envs);
  d.pcg_fric_off = c.take<int>((size_t)pk.n_envs + 1);
  d.pcg_ctl = c.take<unsigned int>(16);
  d.pcg_ritem = c.take<int>((size_t)pk.n_rows / 128);
  d.step_ctl = c.take<unsigned int>(8);
  d.roll_ctl = c.take<unsigned long long>(4);
  d.check_word = c.take<unsigned long long>(2);
  d.q = c.take<double>(R3);
  d.qc = c.take<double>(R3);
  d.pc = c.take<double>(6 * (size_t)pk.n_rows);
  d.pc_acc = c.take<double>(9 * (size_t)pk.n_rows);
  d.body_pc = c.take<double>(144 * (size_t)pk.n_bodies);
  d.body_pc_acc = c.take<double>(144 * (size_t)pk.n_bodies);
  d.body_g = c.take<double>(12 * (size_t)pk.n_bodies);
  d.body_H = c.take<double>(144 * (size_t)pk.n_bodies);
  d.body_E = c.take<double>(pk.n_bodies);
  const size_t hs = d.prec ? sizeof(float) : sizeof(double);
  d.sell_val = c.take<char>(hs * 9 * (size_t)pk.n_sell_blocks);
  d.tetG = c.take<double>(12 * (size_t)pk.n_tets);
  d.tetH = c.take<char>(hs * 144 * (size_t)pk.n_tets);
  d.tetE = c.take<double>(pk.n_tets);
  d.row_E = c.take<double>(pk.n_rows);
  d.cvx = c.take<double>(3 * (size_t)pk.n_cv);
  d.cvp = c.take<double>(3 * (size_t)pk.n_cv);
  d.obj_box = c.take<double>(6 * (size_t)pk.n_obj);
  d.cv_box = c.take<double>(6 * (size_t)pk.n_cv);
  d.tri_box = c.take<double>(6 * (size_t)pk.n_tri);
  d.edge_box = c.take<double>(6 * (size_t)pk.n_edge);
  for (int k = 0; k < 3; ++k) {
    d.bv_cl_box[k] = c.take<double>(6 * (size_t)d.bv_n_cl[k]);
    d.bv_sc_box[k] = c.take<double>(6 * (size_t)d.bv_n_sc[k]);
  }
  {
    // worklist capacity: every query primitive against every smaller object
    long long cap = 0;
    for (const auto& ev : pk.env)
      cap += (long long)(ev.n_cv + ev.n_tri + ev.n_edge) * std::max(1, ev.n_obj - 1);
    d.bp_cap = (int)std::min<long long>(cap, 1LL << 30);
  }
  d.bp_items = c.take<int4>(d.bp_cap);
  d.bp_count = c.take<int>(1);
  d.bp_overflow = c.take<int>(1);
  d.pair_v = c.take<int4>(pk.n_pairs_cap);
  d.pair_kind = c.take<int>(pk.n_pairs_cap);
  d.pair_w = c.take<double>(pk.n_pairs_cap);
  d.pair_eps = c.take<double>(pk.n_pairs_cap);
  d.pair_H = c.take<char>(hs * 78 * ((size_t)pk.n_pairs_cap + 32));
  d.pair_E = c.take<double>(pk.n_pairs_cap);
  d.pair_act = c.take<uint8_t>(pk.n_pairs_cap);
  d.pair_scan = c.take<int>(pk.n_envs + 1);
  d.act_v = c.take<int4>(pk.n_pairs_cap);
  const size_t nfr = prm.friction_mu > 0.0 ? pk.n_pairs_cap : 0;
  d.fr_v = c.take<int4>(nfr);
  d.fr_w = c.take<double>(4 * nfr);
  d.fr_T = c.take<double>(6 * nfr);
  d.fr_rn = c.take<double>(3 * nfr);
  d.fr_ml = c.take<double>(nfr);
  d.fr_S = c.take<double>(6 * nfr);
  d.fr_E = c.take<double>(nfr);
  d.fr_scan = c.take<int>(pk.n_envs + 1);
  d.accd_tail = c.take<int4>(pk.n_pairs_cap);
  d.accd_tail_t = c.take<double>(pk.n_pairs_cap);
  d.accd_tail_ctl = c.take<unsigned int>(2);
  d.cta_part = c.take<double>(4 * (size_t)(pk.n_rows / 128));
  d.env_cnt = c.take<unsigned int>(2 * (size_t)pk.n_envs);
  int mb = 0;
  for (const auto& ev : pk.env) mb = std::max(mb, ev.n_bodies);
  d.max_bodies = mb;
  d.tgt_stage = c.take<double>(12 * (size_t)mb * pk.n_envs);
  d.out_stage = c.take<double>(3 * (size_t)pk.n_coated);
  d.env_s = c.take<double>(NUM_SCALARS * (size_t)pk.n_envs);
  d.env_i = c.take<int>(NUM_INTS * (size_t)pk.n_envs);
}

ipc_status check_env(const ipc_ctx* ctx, int env) {
  if (!ctx || env < 0 || env >= ctx->pk.n_envs) return IPC_EINVAL;
  return IPC_OK;
}

// set the I_SEL column of env_i (and optionally another flag) for a list of envs
ipc_status select_envs(ipc_ctx* ctx, const std::vector<int>& sel, int flag = I_SEL) {
  const int n = ctx->pk.n_envs;
  std::vector<int> col(n, 0);
  for (int e : sel) col[e] = 1;
  CK(cudaMemcpy2DAsync(ctx->dev.env_i + flag, NUM_INTS * sizeof(int), col.data(), sizeof(int), sizeof(int), n,
                       cudaMemcpyHostToDevice, ctx->stream));
  return IPC_OK;
}

ipc_status sync_flags(ipc_ctx* ctx) {
  CK(cudaMemcpyAsync(ctx->h_int, ctx->dev.env_i, NUM_INTS * sizeof(int) * ctx->pk.n_envs, cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaMemcpyAsync(ctx->h_dbl, ctx->dev.env_s, NUM_SCALARS * sizeof(double) * ctx->pk.n_envs,
                     cudaMemcpyDeviceToHost, ctx->stream));
  if (ctx->pcg_graph_pending)
    CK(cudaMemcpyAsync(ctx->h_ctl, ctx->dev.pcg_ctl, 8 * sizeof(unsigned int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->pcg_graph_pending) {
    // the graph ran the WHILE body h_ctl[1] times
    // the graph ran the WHILE body once per launch of iterations
    ctx->launches += (long long)(ctx->h_ctl[1] / (unsigned)pcg_iters_per_launch(ctx->dev, 0xffffffffu)) *
                     ctx->pcg_iter_launches;
    ctx->pcg_graph_pending = false;
  }
  prof_flush(ctx);
  return IPC_OK;
}

int count_flag(const ipc_ctx* ctx, int flag) {
  int c = 0;
  for (int e = 0; e < ctx->pk.n_envs; ++e) c += ctx->h_int[e * NUM_INTS + flag] != 0;
  return c;
}

ipc_status last_cuda(ipc_ctx* ctx) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ctx->err = std::string("kernel launch: ") + cudaGetErrorString(e);
    return IPC_ECUDA;
  }
  return IPC_OK;
}

// ---- the assembled Newton system at the current iterate of active envs,
// on stream s.  The lagged friction records are taken only in the first
// Newton iteration of a step (decided on the device).
ipc_status assemble_system(ipc_ctx* ctx, cudaStream_t s) {
  const Dev& d = ctx->dev;
  KL(ctx, KC_CVPOS, [&] { return launch_cv_pos(d, I_NEWT, false, s); }, s);
  KL(ctx, KC_OBJBOX, [&] { return launch_obj_box(d, I_NEWT, false, s); }, s);
  KL(ctx, KC_MISC, [&] { return launch_env_reset(d, 2, s); }, s);
  KL(ctx, KC_BROAD, [&] { return launch_broad(d, I_NEWT, false, s); }, s);
  KL(ctx, KC_MISC, [&] { return launch_check_overflow(d, s); }, s);
  // barrier terms (side stream 0) and ABD terms (side stream 1) are few,
  // latency-bound threads; they are issued first, at high priority, and run
  // beside the per-tet kernel, which fills the rest of the GPU
  fork_side(ctx, s);
  cudaStream_t s0 = side_of(ctx, s, 0), s1 = side_of(ctx, s, 1);
  KL(ctx, KC_BARRIER, [&] { return launch_fric_setup(d, s0); }, s0);
  KL(ctx, KC_BARRIER, [&] { return launch_barrier(d, I_NEWT, s0); }, s0);
  KL(ctx, KC_BARRIER, [&] { return launch_fric_assemble(d, s0); }, s0);
  KL(ctx, KC_BODY, [&] { return launch_body(d, s1); }, s1);
  KL(ctx, KC_TET, [&] { return launch_tet(d, s); }, s);
  join_side(ctx, s);
  KL(ctx, KC_ASSEMBLE, [&] { return launch_assemble(d, s); }, s);
  KL(ctx, KC_GRAD, [&] { return launch_grad(d, s); }, s);
  KL(ctx, KC_PRECOND, [&] { return launch_precond(d, s); }, s);
  return last_cuda(ctx);
}

// Newton decision after the solve: |p|_inf, converged / AL update / line search
void newton_decide(ipc_ctx* ctx, cudaStream_t s) {
  const Dev& d = ctx->dev;
  KL(ctx, KC_NEWTON, [&] { return launch_newton_check(d, s); }, s);
  KL(ctx, KC_NEWTON, [&] { return launch_newton_decide(d, s); }, s);
  KL(ctx, KC_NEWTON, [&] { return launch_al_update(d, s); }, s);
}

// CCD-filtered backtracking line search, set-up: swept candidates, ACCD
// (side stream) beside the energy at alpha = 0, which needs only the swept
// pair list; the step length starts from ACCD's bound after the join
void line_search_prep(ipc_ctx* ctx, cudaStream_t s) {
  const Dev& d = ctx->dev;
  KL(ctx, KC_CVPOS, [&] { return launch_cv_pos(d, I_LS, true, s); }, s);
  KL(ctx, KC_OBJBOX, [&] { return launch_obj_box(d, I_LS, true, s); }, s);
  KL(ctx, KC_MISC, [&] { return launch_env_reset(d, 5, s); }, s);
  KL(ctx, KC_BROAD, [&] { return launch_broad(d, I_LS, true, s); }, s);
  KL(ctx, KC_MISC, [&] { return launch_check_overflow(d, s); }, s);
  fork_side(ctx, s, 1);
  cudaStream_t s0 = side_of(ctx, s, 0);
  KL(ctx, KC_ACCD, [&] { return launch_accd(d, s0); }, s0);
  KL(ctx, KC_ENERGY, [&] { return launch_energy(d, 0, 0, s); }, s);
  join_side(ctx, s, 1);
  KL(ctx, KC_LS, [&] { return launch_ls_init(d, s); }, s);
}

// one line-search trial: energy at alpha, accept or halve, apply
void line_search_trial(ipc_ctx* ctx, cudaStream_t s) {
  const Dev& d = ctx->dev;
  KL(ctx, KC_ENERGY, [&] { return launch_energy(d, 1, 1, s); }, s);
  KL(ctx, KC_LS, [&] { return launch_ls_decide(d, s); }, s);
  KL(ctx, KC_LS, [&] { return launch_ls_apply(d, s); }, s);
}

constexpr int kPcgPoll = 16;  // host-driven path: PCG iterations between reads of the live-env count

// one PCG iteration on stream s over the device-side work list; returns the
// launches issued.  use_cond: the update kernel sets the graph condition h.
int pcg_iteration(ipc_ctx* ctx, cudaStream_t s, cudaGraphConditionalHandle h = 0, int use_cond = 0,
                  unsigned window = 0xffffffffu) {
  const Dev& d = ctx->dev;
  long long l0 = ctx->launches;
  if (d.pcg_fused) {
    // the whole iteration (with friction terms) as one persistent kernel
    KL(ctx, KC_PCGITER, [&] { return launch_pcg_iter(d, s, h, use_cond, window); }, s);
    return (int)(ctx->launches - l0);
  }
  // contact terms (side stream) beside the SELL mat-vec: both only read
  // z_k and d_{k-1}
  fork_side(ctx, s, 1);
  cudaStream_t s0 = side_of(ctx, s, 0);
  KL(ctx, KC_PAIRSPMV, [&] { return launch_pcg_pairs(d, s0); }, s0);
  KL(ctx, KC_SPMV, [&] { return launch_pcg_matvec(d, s); }, s);
  join_side(ctx, s, 1);
  KL(ctx, KC_FRICSPMV, [&] { return launch_fric_spmv(d, s); }, s);
  KL(ctx, KC_PCGUPD, [&] { return launch_pcg_update(d, s, h, use_cond, window); }, s);
  return (int)(ctx->launches - l0);
}

// Adds a conditional node of `type` on handle h after everything captured so
// far on the capturing stream s, and continues the capture after it;
// *body receives the node's body graph (to be filled by capture-to-graph).
cudaError_t add_conditional(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                            cudaGraph_t* body) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edges = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &edges, &nd);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  // zero-filled storage: the parameter union has no usable default constructor
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
  std::memset(raw, 0, sizeof(raw));
  cudaGraphNodeParams& prm = *reinterpret_cast<cudaGraphNodeParams*>(raw);
  prm.type = cudaGraphNodeTypeConditional;
  prm.conditional.handle = h;
  prm.conditional.type = type;
  prm.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, g, deps, edges, nd, &prm);
  if (e != cudaSuccess) return e;
  *body = prm.conditional.phGraph_out[0];
  return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// graph of the capturing stream s
cudaError_t capturing_graph(cudaStream_t s, cudaGraph_t* g) {
  cudaStreamCaptureStatus cs;
  return cudaStreamGetCaptureInfo(s, &cs, nullptr, g, nullptr, nullptr, nullptr);
}

// The whole PCG solve as one graph: the work-list kernel sets the condition
// of a WHILE node whose body is one iteration; the update kernel's last CTA
// sets it again after every iteration (1 while an env iterates, 0 once
// every env has stopped, at the latest after pcg_max + 2 iterations).  The
// kernels take the context's device tables by value and every per-solve
// quantity lives in device memory, so the graph is captured once per
// context (and again after ipc_autotune changes a launch shape).
ipc_status capture_pcg(ipc_ctx* ctx) {
  cudaStream_t s = ctx->stream, s_body = ctx->cap[0];
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->err = std::string("PCG graph capture: ") + cudaGetErrorString(e) +
               " (the stream cannot be captured, e.g. the legacy default stream)";
    return IPC_ECUDA;
  }
  const long long l0 = ctx->launches;
  cudaGraph_t g = nullptr, body = nullptr;
  cudaGraphConditionalHandle h = 0;
  e = capturing_graph(s, &g);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g, 0, 0);
  if (e == cudaSuccess) {
    launch_pcg_begin(ctx->dev, s, h, 1);
    e = add_conditional(s, h, cudaGraphCondTypeWhile, &body);
  }
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(s_body, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    ctx->pcg_iter_launches = pcg_iteration(ctx, s_body, h, 1);
    cudaGraph_t b2 = nullptr;
    e = cudaStreamEndCapture(s_body, &b2);
  }
  cudaGraph_t gg = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(s, &gg);
  if (e == cudaSuccess) e = e2;
  ctx->launches = l0;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->pcg_exec, gg, 0);
  if (gg) cudaGraphDestroy(gg);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->pcg_exec = nullptr;
    ctx->err = std::string("PCG graph capture: ") + cudaGetErrorString(e);
    return IPC_ECUDA;
  }
  return IPC_OK;
}

// read Dev::pcg_ctl into pinned memory (synchronises the stream)
ipc_status read_pcg_ctl(ipc_ctx* ctx) {
  CK(cudaMemcpyAsync(ctx->h_ctl, ctx->dev.pcg_ctl, 8 * sizeof(unsigned int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  prof_flush(ctx);
  return IPC_OK;
}

ipc_status run_pcg(ipc_ctx* ctx) {
  const Dev& d = ctx->dev;
  cudaStream_t s = ctx->stream;
  KL(ctx, KC_PCGINIT, [&] { return launch_pcg_init(d, s); });
  const bool graph = ctx->graph_mode == 1 && !ctx->prof_on;
  if (graph) {
    if (!ctx->pcg_exec) {
      ipc_status st = capture_pcg(ctx);
      if (st != IPC_OK) return st;
    }
    CK(cudaGraphLaunch(ctx->pcg_exec, s));
    // launches: the work-list kernel now, the iterations' when the
    // iteration count is read back (sync_flags)
    ctx->launches += 1;
    ctx->pcg_graph_pending = true;
    return last_cuda(ctx);
  }
  KL(ctx, KC_PCGINIT, [&] { return launch_pcg_begin(d, s, 0, 0); });
  // every env stops by itself after at most pcg_max iterations
  for (int it = 0; it < ctx->prm.pcg_max + 1; it += kPcgPoll) {
    for (int i = 0; i < kPcgPoll; i += pcg_iters_per_launch(ctx->dev, 0xffffffffu)) pcg_iteration(ctx, s);
    ipc_status st = read_pcg_ctl(ctx);
    if (st != IPC_OK) return st;
    if (ctx->h_ctl[4] == 0) break;  // no env still iterating
  }
  return last_cuda(ctx);
}

// ---- the whole step as one CUDA graph (ipc_set_graph_mode(ctx, 2))
//
//   predict / targets
//   WHILE (an env is in Newton and fewer than newton_max iterations ran)
//     assembly; PCG: work list, WHILE (an env iterates) { mat-vec, update }
//     Newton decision
//     IF (an env needs a line search)
//       swept candidates, ACCD, energy at 0
//       WHILE (an env is in the line search) { energy at alpha, decide, apply }
//   finalize
//
// Every condition is set on the device (k_flag_cond, the PCG update's last
// CTA), so a step needs no host round trip; every loop is bounded by its
// iteration cap on the device.  Capture streams: cap[0] fills the Newton
// body, cap[1] the PCG and line-search bodies, cap[2] the trial loop.
// Adds a conditional node of `type` on h after what the capturing stream cs
// holds, and captures `fill` into its body on stream bs.
template <class F>
cudaError_t cond_body(cudaStream_t cs, cudaStream_t bs, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType t,
                      F&& fill) {
  cudaGraph_t g = nullptr;
  cudaError_t e = add_conditional(cs, h, t, &g);
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(bs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  e = fill();
  cudaGraph_t g2 = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(bs, &g2);
  return e != cudaSuccess ? e : e2;
}

// One Newton iteration of the envs still iterating, captured on cap[0]:
// assembly, the PCG WHILE (body on cap[1]), the Newton decision, the
// line-search IF (cap[1]) with its trial WHILE (cap[2]).  Launch counts of
// its parts go to *base (once per iteration), *pcg_iter, *ls_prep, *ls_trial.
struct IterLaunches {
  long long base = 0, pcg_iter = 0, ls_prep = 0, ls_trial = 0;
};
cudaError_t capture_newton_iteration(ipc_ctx* ctx, cudaGraphConditionalHandle hP, cudaGraphConditionalHandle hA,
                                     cudaGraphConditionalHandle hL, IterLaunches& L,
                                     unsigned window = 0xffffffffu) {
  const Dev& d = ctx->dev;
  cudaStream_t c0 = ctx->cap[0], c1 = ctx->cap[1], c2 = ctx->cap[2];
  const unsigned lsmax = (unsigned)ctx->prm.ls_max + 1u;
  const long long m = ctx->launches;
  KL(ctx, KC_MISC, [&] { return launch_env_reset(d, 1, c0); }, c0);
  if (assemble_system(ctx, c0) != IPC_OK) return cudaErrorUnknown;
  KL(ctx, KC_PCGINIT, [&] { return launch_pcg_init(d, c0); }, c0);
  KL(ctx, KC_PCGINIT, [&] { return launch_pcg_begin(d, c0, hP, 1); }, c0);
  long long mn = ctx->launches;
  cudaError_t e = cond_body(c0, c1, hP, cudaGraphCondTypeWhile, [&] {
    L.pcg_iter = pcg_iteration(ctx, c1, hP, 1, window);
    return cudaSuccess;
  });
  if (e != cudaSuccess) return e;
  mn = ctx->launches - mn;
  newton_decide(ctx, c0);
  KL(ctx, KC_MISC, [&] { return launch_flag_cond(d, c0, I_LS, 3, -1, -1, 1, 0, hA, 1); }, c0);
  long long ml = ctx->launches;
  e = cond_body(c0, c1, hA, cudaGraphCondTypeIf, [&] {
    long long mp = ctx->launches;
    line_search_prep(ctx, c1);
    KL(ctx, KC_MISC, [&] { return launch_flag_cond(d, c1, I_LS, 3, 6, -1, -1, 0xffffffffu, hL, 1); }, c1);
    L.ls_prep = ctx->launches - mp;
    long long mt = ctx->launches;
    cudaError_t e3 = cond_body(c1, c2, hL, cudaGraphCondTypeWhile, [&] {
      line_search_trial(ctx, c2);
      KL(ctx, KC_MISC, [&] { return launch_flag_cond(d, c2, I_LS, 3, 1, 5, -1, lsmax, hL, 1); }, c2);
      return cudaSuccess;
    });
    L.ls_trial = ctx->launches - mt;
    return e3;
  });
  ml = ctx->launches - ml;
  L.base = ctx->launches - m - mn - ml;
  return e;
}

// ends a capture begun on ctx->stream and instantiates it into *exec
ipc_status finish_capture(ipc_ctx* ctx, cudaError_t e, long long l0, cudaGraphExec_t* exec, const char* what) {
  cudaGraph_t gg = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &gg);
  if (e == cudaSuccess) e = e2;
  ctx->launches = l0;
  if (e == cudaSuccess) e = cudaGraphInstantiate(exec, gg, 0);
  if (gg) cudaGraphDestroy(gg);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *exec = nullptr;
    ctx->err = std::string(what) + ": " + cudaGetErrorString(e);
    return IPC_ECUDA;
  }
  return IPC_OK;
}

cudaError_t begin_capture(ipc_ctx* ctx, const char* what) {
  cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->err = std::string(what) + ": " + cudaGetErrorString(e) +
               " (the stream cannot be captured, e.g. the legacy default stream)";
  }
  return e;
}

ipc_status capture_step(ipc_ctx* ctx) {
  const Dev& d = ctx->dev;
  cudaStream_t s = ctx->stream;
  if (begin_capture(ctx, "step graph capture") != cudaSuccess) return IPC_ECUDA;
  const long long l0 = ctx->launches;
  ipc_ctx::StepLaunches& L = ctx->step_launches;
  L = ipc_ctx::StepLaunches{};
  cudaGraph_t root = nullptr;
  cudaGraphConditionalHandle hN = 0, hP = 0, hA = 0, hL = 0;
  cudaError_t e = capturing_graph(s, &root);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hN, root, 0, 0);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hP, root, 0, 0);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hA, root, 0, 0);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hL, root, 0, 0);
  const unsigned nmax = (unsigned)ctx->prm.newton_max;
  cudaStream_t c0 = ctx->cap[0];
  if (e == cudaSuccess) {
    long long m = ctx->launches;
    KL(ctx, KC_MISC, [&] { return launch_env_reset(d, 0, s); }, s);
    KL(ctx, KC_PREDICT, [&] { return launch_predict(d, I_SEL, s); }, s);
    KL(ctx, KC_PREDICT, [&] { return launch_attach_targets(d, I_SEL, s); }, s);
    KL(ctx, KC_MISC, [&] { return launch_flag_cond(d, s, I_ACTIVE, 2, -1, -1, -1, 0, hN, 1); }, s);
    L.pre = ctx->launches - m;
  }
  if (e == cudaSuccess)
    e = cond_body(s, c0, hN, cudaGraphCondTypeWhile, [&] {
      IterLaunches it;
      cudaError_t e1 = capture_newton_iteration(ctx, hP, hA, hL, it);
      long long m = ctx->launches;
      KL(ctx, KC_MISC, [&] { return launch_flag_cond(d, c0, I_ACTIVE, 2, 0, -1, -1, nmax, hN, 1); }, c0);
      L.newton = it.base + (ctx->launches - m);
      L.pcg_iter = it.pcg_iter;
      L.ls_prep = it.ls_prep;
      L.ls_trial = it.ls_trial;
      return e1;
    });
  if (e == cudaSuccess) {
    long long m = ctx->launches;
    KL(ctx, KC_MISC, [&] { return launch_finalize(d, s); }, s);
    L.post = ctx->launches - m;
  }
  return finish_capture(ctx, e, l0, &ctx->step_exec, "step graph capture");
}

// ---- a rollout as one CUDA graph (ipc_rollout)
//
//   every selected env begins step 0
//   WHILE (an env runs or begins a step, below the loop cap)
//     envs beginning a step: targets of their step, counters, predict
//     one Newton iteration of the envs inside a step (as in the step graph)
//     envs whose step ended: Newton cap, finalize, counters, next step
//
// The table address, the step count and the cap live in device memory
// (k_roll_setup before each launch), so the graph is captured once.
ipc_status capture_roll(ipc_ctx* ctx) {
  const Dev& d = ctx->dev;
  cudaStream_t s = ctx->stream;
  if (begin_capture(ctx, "rollout graph capture") != cudaSuccess) return IPC_ECUDA;
  const long long l0 = ctx->launches;
  ipc_ctx::RollLaunches& L = ctx->roll_launches;
  L = ipc_ctx::RollLaunches{};
  cudaGraph_t root = nullptr;
  cudaGraphConditionalHandle hR = 0, hP = 0, hA = 0, hL = 0;
  cudaError_t e = capturing_graph(s, &root);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hR, root, 0, 0);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hP, root, 0, 0);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hA, root, 0, 0);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hL, root, 0, 0);
  cudaStream_t c0 = ctx->cap[0];
  if (e == cudaSuccess) {
    long long m = ctx->launches;
    KL(ctx, KC_MISC, [&] { return launch_roll_init(d, s); }, s);
    KL(ctx, KC_MISC, [&] { return launch_roll_cond(d, s, hR); }, s);
    L.pre = ctx->launches - m;
  }
  if (e == cudaSuccess)
    e = cond_body(s, c0, hR, cudaGraphCondTypeWhile, [&] {
      long long m = ctx->launches;
      KL(ctx, KC_PREDICT, [&] { return launch_roll_begin(d, c0); }, c0);
      IterLaunches it;
      const int w = ctx->prm.rollout_pcg_window;
      cudaError_t e1 = capture_newton_iteration(ctx, hP, hA, hL, it, w > 0 ? (unsigned)w : 0xffffffffu);
      KL(ctx, KC_MISC, [&] { return launch_roll_end(d, c0); }, c0);
      KL(ctx, KC_MISC, [&] { return launch_roll_cond(d, c0, hR); }, c0);
      L.iter = (ctx->launches - m) - it.pcg_iter - it.ls_prep - it.ls_trial;
      L.pcg_iter = it.pcg_iter;
      L.ls_prep = it.ls_prep;
      L.ls_trial = it.ls_trial;
      return e1;
    });
  return finish_capture(ctx, e, l0, &ctx->roll_exec, "rollout graph capture");
}

// One Newton iteration of the envs still iterating, driven from the host
// (plain launches; the flags are read back after the decision and after
// every line-search trial).
ipc_status newton_iteration_host(ipc_ctx* ctx) {
  const Dev& d = ctx->dev;
  cudaStream_t s = ctx->stream;
  ipc_status st;
  KL(ctx, KC_MISC, [&] { return launch_env_reset(d, 1, s); });
  if ((st = assemble_system(ctx, s)) != IPC_OK) return st;
  if ((st = run_pcg(ctx)) != IPC_OK) return st;
  newton_decide(ctx, s);
  if ((st = sync_flags(ctx)) != IPC_OK) return st;
  if (count_flag(ctx, I_LS) > 0) {
    line_search_prep(ctx, s);
    for (int ls = 0; ls < ctx->prm.ls_max; ++ls) {
      line_search_trial(ctx, s);
      if ((st = sync_flags(ctx)) != IPC_OK) return st;
      if (count_flag(ctx, I_LS) == 0) break;
    }
  }
  return IPC_OK;
}

// drop captured graphs (launch shapes or modes changed)
void drop_graphs(ipc_ctx* ctx) {
  if (ctx->pcg_exec) cudaGraphExecDestroy(ctx->pcg_exec);
  if (ctx->step_exec) cudaGraphExecDestroy(ctx->step_exec);
  if (ctx->roll_exec) cudaGraphExecDestroy(ctx->roll_exec);
  ctx->pcg_exec = nullptr;
  ctx->step_exec = nullptr;
  ctx->roll_exec = nullptr;
}

// user-order DoF vector <-> row space of one env
void dof_to_rows(const ipc_ctx* ctx, int env, const double* dof, std::vector<double>& rows) {
  const EnvInfo& ev = ctx->pk.env[env];
  rows.assign(3 * (size_t)ev.n_rows, 0.0);
  for (int r = 0; r < ev.n_verts; ++r)
    for (int c = 0; c < 3; ++c) rows[3 * r + c] = dof[3 * ev.perm[r] + c];
  for (int b = 0; b < ev.n_bodies; ++b)
    for (int k = 0; k < 12; ++k) rows[3 * (ev.gel_rows + 4 * b) + k] = dof[3 * ev.n_verts + 12 * b + k];
}
void rows_to_dof(const ipc_ctx* ctx, int env, const std::vector<double>& rows, double* dof) {
  const EnvInfo& ev = ctx->pk.env[env];
  for (int r = 0; r < ev.n_verts; ++r)
    for (int c = 0; c < 3; ++c) dof[3 * ev.perm[r] + c] = rows[3 * r + c];
  for (int b = 0; b < ev.n_bodies; ++b)
    for (int k = 0; k < 12; ++k) dof[3 * ev.n_verts + 12 * b + k] = rows[3 * (ev.gel_rows + 4 * b) + k];
}

ipc_status upload_rows(ipc_ctx* ctx, int env, double* dst, const std::vector<double>& rows) {
  const EnvInfo& ev = ctx->pk.env[env];
  CK(cudaMemcpyAsync(dst + 3 * (size_t)ev.row_begin, rows.data(), rows.size() * sizeof(double),
                     cudaMemcpyHostToDevice, ctx->stream));
  return IPC_OK;
}
ipc_status download_rows(ipc_ctx* ctx, int env, const double* src, std::vector<double>& rows) {
  const EnvInfo& ev = ctx->pk.env[env];
  rows.resize(3 * (size_t)ev.n_rows);
  CK(cudaMemcpyAsync(rows.data(), src + 3 * (size_t)ev.row_begin, rows.size() * sizeof(double),
                     cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return IPC_OK;
}

// prepare one env as if a step starts (selection, prediction, targets)
ipc_status begin_single(ipc_ctx* ctx, int env) {
  ipc_status st = select_envs(ctx, {env});
  if (st != IPC_OK) return st;
  KL(ctx, KC_MISC, [&] { return launch_env_reset(ctx->dev, 0, ctx->stream); });
  KL(ctx, KC_PREDICT, [&] { return launch_predict(ctx->dev, I_SEL, ctx->stream); });
  KL(ctx, KC_PREDICT, [&] { return launch_attach_targets(ctx->dev, I_SEL, ctx->stream); });
  KL(ctx, KC_MISC, [&] { return launch_env_reset(ctx->dev, 1, ctx->stream); });
  return last_cuda(ctx);
}

// Time `reps` launches of f on the ctx stream (events), after one warm-up.
template <class F>
ipc_status time_launches(ipc_ctx* ctx, int reps, F&& f, float* us) {
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  f();
  CK(cudaEventRecord(a, ctx->stream));
  for (int i = 0; i < reps; ++i) f();
  CK(cudaEventRecord(b, ctx->stream));
  CK(cudaEventSynchronize(b));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *us = 1e3f * ms / (float)reps;
  return last_cuda(ctx);
}

}  // namespace

extern "C" {

void ipc_default_params(ipc_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->dt = 1e-3;
  p->gravity[0] = 0.0; p->gravity[1] = 0.0; p->gravity[2] = -9.81;
  p->dhat = 1e-4;
  p->kappa = 1e6;
  p->newton_tol = 1e-4;
  p->pcg_rel_tol = 1e-4;
  p->newton_max = 300;
  p->pcg_max = 1000;
  p->ls_max = 30;
  p->accd_max = 10000;
  p->accd_s = 0.1;
  p->al_kappa = 1e6;
  p->al_max = 10;
  p->ee_mollifier = 1e-3;
  p->precision = 0;
  p->max_pairs_per_env = 0;
  p->friction_mu = 0.0;
  p->friction_eps_v = 1e-3;
  p->newton_abs_after = 1000000;
  p->rollout_pcg_window = 0;
  p->pcg_fused = 1;
  p->pcg_iters_per_launch = 8;
}

ipc_status ipc_workspace_bytes(const ipc_scene_desc* scenes, int n_envs, const ipc_params* prm, size_t* bytes) {
  if (!prm || !bytes) return IPC_EINVAL;
  Pack pk;
  std::string err;
  if (!build_pack(scenes, n_envs, *prm, pk, err)) return IPC_EINVAL;
  Carver c{nullptr};
  Dev d;
  Extra ex;
  std::vector<std::pair<const void*, std::pair<void*, size_t>>> up;
  carve(pk, *prm, c, d, ex, up);
  *bytes = c.off;
  return IPC_OK;
}

ipc_status ipc_create_envs(const ipc_scene_desc* scenes, int n_envs, const ipc_params* prm, void* dev_workspace,
                           size_t ws_bytes, void* cuda_stream, ipc_ctx** out) {
  if (!prm || !out || !dev_workspace) return IPC_EINVAL;
  if (prm->dt <= 0 || prm->dhat <= 0 || prm->kappa <= 0 || prm->newton_max < 1 || prm->pcg_max < 1 ||
      prm->newton_abs_after < 0 || prm->rollout_pcg_window < 0 || prm->rollout_pcg_window == 1 ||
      (prm->rollout_pcg_window & 1) || prm->pcg_fused < 0 || prm->pcg_fused > 2 ||
      prm->pcg_iters_per_launch < 1 || prm->pcg_iters_per_launch > 16 ||
      prm->ls_max < 1 || prm->accd_max < 1 || !(prm->accd_s > 0 && prm->accd_s < 1))
    return IPC_EINVAL;
  if (reinterpret_cast<uintptr_t>(dev_workspace) % 256 != 0) return IPC_EINVAL;
  ipc_ctx* ctx = new ipc_ctx();
  ctx->prm = *prm;
  ctx->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  if (!build_pack(scenes, n_envs, *prm, ctx->pk, ctx->err)) {
    *out = ctx;  // carries the message
    return IPC_EINVAL;
  }
  Carver c{reinterpret_cast<char*>(dev_workspace)};
  Extra ex;
  std::vector<std::pair<const void*, std::pair<void*, size_t>>> up;
  carve(ctx->pk, *prm, c, ctx->dev, ex, up);
  if (c.off > ws_bytes) {
    ctx->err = "workspace too small";
    *out = ctx;
    return IPC_ENOMEM;
  }
  ctx->ws = reinterpret_cast<char*>(dev_workspace);
  ctx->ws_bytes = ws_bytes;
  *out = ctx;
  // the device the context's stream (and workspace) belong to
  if (ctx->stream) CK(cudaStreamGetDevice(ctx->stream, &ctx->device));
  else CK(cudaGetDevice(&ctx->device));
  const Pack& pk = ctx->pk;
  for (auto& u : up) CK(cudaMemcpyAsync(u.second.first, u.first, u.second.second, cudaMemcpyHostToDevice, ctx->stream));
  // zero every dynamic array (from x to the end of the workspace)
  char* dyn0 = reinterpret_cast<char*>(ctx->dev.x);
  CK(cudaMemsetAsync(dyn0, 0, (ctx->ws + c.off) - dyn0, ctx->stream));
  size_t R3 = 3 * (size_t)pk.n_rows * sizeof(double);
  CK(cudaMemcpyAsync(ctx->dev.x, pk.rest_x.data(), R3, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->dev.s_tgt, pk.rest_x.data(), R3, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMallocHost(&ctx->h_int, NUM_INTS * sizeof(int) * (size_t)pk.n_envs));
  CK(cudaMallocHost(&ctx->h_dbl, NUM_SCALARS * sizeof(double) * (size_t)pk.n_envs));
  CK(cudaMallocHost(&ctx->h_ctl, 8 * sizeof(unsigned int)));
  CK(cudaMallocHost(&ctx->h_step_ctl, 8 * sizeof(unsigned int)));
  for (const auto& ev : pk.env) ctx->max_bodies = std::max(ctx->max_bodies, ev.n_bodies);
  int prio_least = 0, prio_greatest = 0;
  CK(cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest));
  for (int i = 0; i < 2; ++i) {
    for (int k = 0; k < 4; ++k) {
      CK(cudaStreamCreateWithPriority(&ctx->side[k][i], cudaStreamNonBlocking, prio_greatest));
      CK(cudaEventCreateWithFlags(&ctx->ev_join[k][i], cudaEventDisableTiming));
    }
  }
  for (int k = 0; k < 4; ++k) CK(cudaEventCreateWithFlags(&ctx->ev_fork[k], cudaEventDisableTiming));
  for (int i = 0; i < 3; ++i) CK(cudaStreamCreateWithFlags(&ctx->cap[i], cudaStreamNonBlocking));
  // persistent PCG grid: every resident CTA of the two PCG kernels
  CK(cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, ctx->device));
  ctx->dev.pcg_grid = ctx->n_sm * pcg_ctas_per_sm(ctx->dev.prec, ctx->dev.spmv_unroll);
  ctx->dev.pcg_grid_fused =
      ctx->n_sm * pcg_iter_ctas_per_sm(ctx->dev.prec, ctx->dev.spmv_unroll, ctx->dev.pcg_iter_bound, ctx->dev.fr_mu > 0.0);
  ctx->dev.pcg_grid_multi = ctx->n_sm * pcg_multi_ctas_per_sm(ctx->dev.prec, ctx->dev.spmv_unroll, ctx->dev.fr_mu > 0.0);
  ctx->dev.pcg_grid_pairs = ctx->n_sm * 4;
  CK(cudaMemsetAsync(ctx->dev.check_word, 0, 2 * sizeof(unsigned long long), ctx->stream));
  CK(cudaMemsetAsync(ctx->dev.pcg_ritem, 0xff, sizeof(int) * (size_t)(ctx->pk.n_rows / 128), ctx->stream));
  ctx->dev.pairs_grid = ctx->n_sm * 8;
  CK(cudaStreamSynchronize(ctx->stream));
  return IPC_OK;
}

ipc_status ipc_destroy(ipc_ctx* ctx) {
  if (!ctx) return IPC_EINVAL;
  if (ctx->h_int) cudaFreeHost(ctx->h_int);
  if (ctx->h_dbl) cudaFreeHost(ctx->h_dbl);
  if (ctx->h_ctl) cudaFreeHost(ctx->h_ctl);
  if (ctx->h_step_ctl) cudaFreeHost(ctx->h_step_ctl);
  for (int i = 0; i < 3; ++i)
    if (ctx->cap[i]) cudaStreamDestroy(ctx->cap[i]);
  drop_graphs(ctx);
  for (auto& pe : ctx->pending) { cudaEventDestroy(pe.a); cudaEventDestroy(pe.b); }
  for (auto e : ctx->ev_free) cudaEventDestroy(e);
  for (int i = 0; i < 2; ++i) {
    for (int k = 0; k < 4; ++k) {
      if (ctx->side[k][i]) cudaStreamDestroy(ctx->side[k][i]);
      if (ctx->ev_join[k][i]) cudaEventDestroy(ctx->ev_join[k][i]);
    }
  }
  for (int k = 0; k < 4; ++k)
    if (ctx->ev_fork[k]) cudaEventDestroy(ctx->ev_fork[k]);
  delete ctx;
  return IPC_OK;
}

const char* ipc_last_error(const ipc_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

ipc_status ipc_set_graph_mode(ipc_ctx* ctx, int mode) {
  if (!ctx || mode < 0 || mode > 2) return IPC_EINVAL;
  if (mode != ctx->graph_mode) drop_graphs(ctx);
  ctx->graph_mode = mode;
  return IPC_OK;
}

ipc_status ipc_autotune(ipc_ctx* ctx, int reps, ipc_tuning* out) {
  if (!ctx || reps <= 0) return IPC_EINVAL;
  Dev& d = ctx->dev;
  cudaStream_t s = ctx->stream;
  ipc_status st;
  if (ctx->pk.n_envs <= 0) return IPC_EINVAL;
  // The mat-vec shapes are timed on two PCG batches, every env and every
  // fourth env (a solve's launches shrink as envs converge), and judged on
  // the mean of the two.  The mat-vec only writes PCG scratch (q, the new
  // direction buffer, the d.q sums) and the contact accumulator, which is
  // cleared afterwards.
  std::vector<int> all(ctx->pk.n_envs), quarter;
  for (int e = 0; e < ctx->pk.n_envs; ++e) {
    all[e] = e;
    if (e % 4 == 0) quarter.push_back(e);
  }
  auto time_matvec = [&](float* us) -> ipc_status {
    float a = 0.f, q = 0.f;
    ipc_status r;
    if ((r = select_envs(ctx, all, I_PCG)) != IPC_OK) return r;
    launch_pcg_begin(d, s, 0, 0);
    if ((r = time_launches(ctx, reps, [&] { launch_pcg_matvec(d, s); }, &a)) != IPC_OK) return r;
    if ((r = select_envs(ctx, quarter, I_PCG)) != IPC_OK) return r;
    launch_pcg_begin(d, s, 0, 0);
    if ((r = time_launches(ctx, reps, [&] { launch_pcg_matvec(d, s); }, &q)) != IPC_OK) return r;
    *us = 0.5f * (a + q);
    return IPC_OK;
  };
  ipc_tuning t{};
  // a candidate replaces the default shape only when it is more than 5%
  // faster (ties and noise keep the default)
  const int us_[3] = {2, 4, 8};
  const int def_u = 2;
  for (int k = 0; k < 3; ++k) {
    d.spmv_unroll = us_[k];
    d.pcg_grid = ctx->n_sm * pcg_ctas_per_sm(d.prec, us_[k]);
    if ((st = time_matvec(&t.spmv_us[k])) != IPC_OK) return st;
  }
  const float def_spmv = t.spmv_us[def_u == 2 ? 0 : 1];
  int best_u = def_u;
  float best = def_spmv;
  for (int k = 0; k < 3; ++k)
    if (t.spmv_us[k] < best && t.spmv_us[k] < 0.95f * def_spmv) { best = t.spmv_us[k]; best_u = us_[k]; }
  d.spmv_unroll = best_u;
  // persistent grid: half, all or twice the resident CTAs per SM
  const int occ = pcg_ctas_per_sm(d.prec, best_u);
  const int cand[3] = {occ > 1 ? occ / 2 : 1, occ, 2 * occ};
  for (int k = 0; k < 3; ++k) {
    d.pcg_grid = ctx->n_sm * cand[k];
    if ((st = time_matvec(&t.grid_us[k])) != IPC_OK) return st;
  }
  int best_c = occ;
  best = t.grid_us[1];
  for (int k = 0; k < 3; ++k)
    if (t.grid_us[k] < best && t.grid_us[k] < 0.95f * t.grid_us[1]) { best = t.grid_us[k]; best_c = cand[k]; }
  d.pcg_grid = ctx->n_sm * best_c;
  CK(cudaMemsetAsync(d.qc, 0, 3 * sizeof(double) * (size_t)d.n_rows, s));
  if ((st = select_envs(ctx, {}, I_PCG)) != IPC_OK) return st;
  // the fused iteration kernel, register bound on (default) or off: PCG
  // iterations from a fresh start (p = 0, r = -g, z = P^-1 r: the PCG
  // scratch of the last Newton iteration's system), on every env and on
  // every fourth env, the mean time per iteration; converging envs leave
  // as in a real solve.  The flags the solve sets (I_PCG, I_DEC) are
  // cleared afterwards; the next step's start resets the counters.
  auto time_fused = [&](float* us) -> ipc_status {
    float a = 0.f, q = 0.f;
    ipc_status r;
    for (int pass = 0; pass < 2; ++pass) {
      if ((r = select_envs(ctx, {}, I_PCG)) != IPC_OK) return r;
      if ((r = select_envs(ctx, pass ? quarter : all, I_NEWT)) != IPC_OK) return r;
      launch_pcg_init(d, s);
      launch_pcg_begin(d, s, 0, 0);
      if ((r = time_launches(ctx, reps, [&] { launch_pcg_iter(d, s, 0, 0, 0xffffffffu); }, pass ? &q : &a)) !=
          IPC_OK)
        return r;
    }
    *us = 0.5f * (a + q);
    return IPC_OK;
  };
  int best_b = 1;
  if (d.pcg_fused) {
    // the bound applies to the single-iteration kernel (k_pcg_iter: one
    // iteration per launch, inside rollout windows), so that is what is timed
    const int multi = d.pcg_multi;
    d.pcg_multi = 1;
    for (int b = 1; b >= 0; --b) {
      d.pcg_iter_bound = b;
      d.pcg_grid_fused = ctx->n_sm * pcg_iter_ctas_per_sm(d.prec, d.spmv_unroll, b, d.fr_mu > 0.0);
      if ((st = time_fused(&t.pcg_iter_us[1 - b])) != IPC_OK) {
        d.pcg_multi = multi;
        return st;
      }
    }
    d.pcg_multi = multi;
    if (t.pcg_iter_us[1] < 0.95f * t.pcg_iter_us[0]) best_b = 0;
    CK(cudaMemsetAsync(d.qc, 0, 3 * sizeof(double) * (size_t)d.n_rows, s));
    if ((st = select_envs(ctx, {}, I_NEWT)) != IPC_OK) return st;
    if ((st = select_envs(ctx, {}, I_PCG)) != IPC_OK) return st;
    if ((st = select_envs(ctx, {}, I_DEC)) != IPC_OK) return st;
  }
  d.pcg_iter_bound = best_b;
  d.pcg_grid_fused = ctx->n_sm * pcg_iter_ctas_per_sm(d.prec, d.spmv_unroll, best_b, d.fr_mu > 0.0);
  d.pcg_grid_multi = ctx->n_sm * pcg_multi_ctas_per_sm(d.prec, d.spmv_unroll, d.fr_mu > 0.0);
  // gather assembly: 64, 128 or 256 threads per CTA, every env counted as
  // starting a Newton iteration (rewrites the SELL values from the stored
  // element blocks)
  if ((st = select_envs(ctx, all, I_NEWT)) != IPC_OK) return st;
  const int asm_cand[3] = {64, 128, 256};
  for (int k = 0; k < 3; ++k) {
    d.asm_block = asm_cand[k];
    if ((st = time_launches(ctx, reps, [&] { launch_assemble(d, s); }, &t.assemble_us[k])) != IPC_OK) return st;
  }
  int best_a = 128;
  best = t.assemble_us[1];
  for (int k = 0; k < 3; ++k)
    if (t.assemble_us[k] < best && t.assemble_us[k] < 0.95f * t.assemble_us[1]) { best = t.assemble_us[k]; best_a = asm_cand[k]; }
  d.asm_block = best_a;
  if ((st = select_envs(ctx, {}, I_NEWT)) != IPC_OK) return st;
  // candidate-pair search: 4, 8 or 16 CTAs per SM over every env's current
  // positions (the lists are rebuilt at the next Newton iteration)
  if ((st = select_envs(ctx, all)) != IPC_OK) return st;
  const int pc_cand[3] = {4, 8, 16};
  for (int k = 0; k < 3; ++k) {
    d.pairs_grid = ctx->n_sm * pc_cand[k];
    if ((st = time_launches(ctx, reps, [&] {
           launch_env_reset(d, 6, s);
           launch_broad(d, I_SEL, false, s);
         }, &t.pairs_us[k])) != IPC_OK)
      return st;
  }
  int best_p = 8;
  best = t.pairs_us[1];
  for (int k = 0; k < 3; ++k)
    if (t.pairs_us[k] < best && t.pairs_us[k] < 0.95f * t.pairs_us[1]) { best = t.pairs_us[k]; best_p = pc_cand[k]; }
  d.pairs_grid = ctx->n_sm * best_p;
  t.assemble_block = best_a;
  t.pairs_ctas_per_sm = best_p;
  CK(cudaStreamSynchronize(s));
  // the captured graphs hold the old launch shapes
  drop_graphs(ctx);
  t.spmv_unroll = best_u;
  t.pcg_ctas_per_sm = best_c;
  for (int k = 0; k < 3; ++k) t.grid_ctas_per_sm[k] = cand[k];
  t.pcg_iter_bound = best_b;
  if (out) *out = t;
  return IPC_OK;
}

int ipc_num_envs(const ipc_ctx* ctx) { return ctx ? ctx->pk.n_envs : 0; }

ipc_status ipc_check_report(ipc_ctx* ctx, int* checks_built, int* code, long long* index) {
  if (!ctx) return IPC_EINVAL;
#ifdef IPC_CHECKS
  if (checks_built) *checks_built = 1;
#else
  if (checks_built) *checks_built = 0;
#endif
  unsigned long long w[2] = {0, 0};
  CK(cudaMemcpyAsync(w, ctx->dev.check_word, sizeof(w), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (code) *code = (int)w[0];
  if (index) *index = (long long)w[1];
  return IPC_OK;
}

ipc_status ipc_env_sizes(const ipc_ctx* ctx, int env, int* n_verts, int* n_bodies, int* n_surface_out) {
  if (check_env(ctx, env) != IPC_OK) return IPC_EINVAL;
  const EnvInfo& ev = ctx->pk.env[env];
  if (n_verts) *n_verts = ev.n_verts;
  if (n_bodies) *n_bodies = ev.n_bodies;
  if (n_surface_out) *n_surface_out = ev.n_coated;
  return IPC_OK;
}

ipc_status ipc_body_com(const ipc_ctx* ctx, int env, int body, double com[3]) {
  if (check_env(ctx, env) != IPC_OK || !com) return IPC_EINVAL;
  const EnvInfo& ev = ctx->pk.env[env];
  if (body < 0 || body >= ev.n_bodies) return IPC_EINVAL;
  for (int k = 0; k < 3; ++k) com[k] = ev.body_com[3 * body + k];
  return IPC_OK;
}

ipc_status ipc_get_state(ipc_ctx* ctx, int env, double* x, double* v, double* y, double* ydot) {
  if (check_env(ctx, env) != IPC_OK) return IPC_EINVAL;
  const EnvInfo& ev = ctx->pk.env[env];
  std::vector<double> rows;
  std::vector<double> dof(3 * (size_t)ev.n_verts + 12 * (size_t)ev.n_bodies);
  for (int which = 0; which < 2; ++which) {
    double* gx = which == 0 ? x : v;
    double* gy = which == 0 ? y : ydot;
    if (!gx && !gy) continue;
    ipc_status st = download_rows(ctx, env, which == 0 ? ctx->dev.x : ctx->dev.v, rows);
    if (st != IPC_OK) return st;
    rows_to_dof(ctx, env, rows, dof.data());
    if (gx) std::memcpy(gx, dof.data(), 3 * sizeof(double) * ev.n_verts);
    if (gy) std::memcpy(gy, dof.data() + 3 * ev.n_verts, 12 * sizeof(double) * ev.n_bodies);
  }
  return IPC_OK;
}

ipc_status ipc_set_state(ipc_ctx* ctx, int env, const double* x, const double* v, const double* y,
                         const double* ydot) {
  if (check_env(ctx, env) != IPC_OK) return IPC_EINVAL;
  const EnvInfo& ev = ctx->pk.env[env];
  size_t nd = 3 * (size_t)ev.n_verts + 12 * (size_t)ev.n_bodies;
  // non-finite input is rejected before anything is uploaded
  auto finite = [](const double* a, size_t n) {
    for (size_t i = 0; i < n; ++i)
      if (!std::isfinite(a[i])) return false;
    return true;
  };
  const size_t nx = 3 * (size_t)ev.n_verts, ny = 12 * (size_t)ev.n_bodies;
  if ((x && !finite(x, nx)) || (v && !finite(v, nx)) || (y && !finite(y, ny)) || (ydot && !finite(ydot, ny))) {
    ctx->err = "set_state: non-finite input";
    return IPC_EINVAL;
  }
  std::vector<double> old_x, old_v, dof(nd), rows;
  ipc_status st;
  if ((st = download_rows(ctx, env, ctx->dev.x, old_x)) != IPC_OK) return st;
  if ((st = download_rows(ctx, env, ctx->dev.v, old_v)) != IPC_OK) return st;
  for (int which = 0; which < 2; ++which) {
    const double* gx = which == 0 ? x : v;
    const double* gy = which == 0 ? y : ydot;
    if (!gx && !gy) continue;
    rows_to_dof(ctx, env, which == 0 ? old_x : old_v, dof.data());
    if (gx) std::memcpy(dof.data(), gx, 3 * sizeof(double) * ev.n_verts);
    if (gy) std::memcpy(dof.data() + 3 * ev.n_verts, gy, 12 * sizeof(double) * ev.n_bodies);
    dof_to_rows(ctx, env, dof.data(), rows);
    // keep padding rows as they were
    const std::vector<double>& old = which == 0 ? old_x : old_v;
    for (int r = ev.n_verts; r < ev.n_rows; ++r)
      if (r < ev.gel_rows || r >= ev.gel_rows + 4 * ev.n_bodies)
        for (int c = 0; c < 3; ++c) rows[3 * r + c] = old[3 * r + c];
    if ((st = upload_rows(ctx, env, which == 0 ? ctx->dev.x : ctx->dev.v, rows)) != IPC_OK) return st;
  }
  // feasibility: no inverted tet, no touching pair
  if ((st = select_envs(ctx, {env})) != IPC_OK) return st;
  KL(ctx, KC_MISC, [&] { return launch_env_reset(ctx->dev, 3, ctx->stream); });
  KL(ctx, KC_MISC, [&] { return launch_check_inverted(ctx->dev, ctx->stream); });
  KL(ctx, KC_CVPOS, [&] { return launch_cv_pos(ctx->dev, I_SEL, false, ctx->stream); });
  KL(ctx, KC_OBJBOX, [&] { return launch_obj_box(ctx->dev, I_SEL, false, ctx->stream); });
  KL(ctx, KC_MISC, [&] { return launch_env_reset(ctx->dev, 6, ctx->stream); });
  KL(ctx, KC_BROAD, [&] { return launch_broad(ctx->dev, I_SEL, false, ctx->stream); });
  KL(ctx, KC_MISC, [&] { return launch_cross_check(ctx->dev, I_SEL, ctx->stream); });
  KL(ctx, KC_MISC, [&] { return launch_min_dist(ctx->dev, I_SEL, ctx->stream); });
  if ((st = last_cuda(ctx)) != IPC_OK) return st;
  if ((st = sync_flags(ctx)) != IPC_OK) return st;
  ipc_status verdict = IPC_OK;
  const int flag = ctx->h_int[env * NUM_INTS + I_FLAG];
  if (flag == 1) verdict = IPC_EINVERTED;
  else if (flag == 2 || !(ctx->h_dbl[env * NUM_SCALARS + S_MIND] > 0.0)) verdict = IPC_EINTERSECT;
  if (verdict != IPC_OK) {
    upload_rows(ctx, env, ctx->dev.x, old_x);
    upload_rows(ctx, env, ctx->dev.v, old_v);
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->err = verdict == IPC_EINVERTED ? "set_state: inverted tetrahedron"
               : flag == 2             ? "set_state: surfaces cross (an edge passes through a triangle)"
                                       : "set_state: surfaces touch";
  }
  return verdict;
}

ipc_status ipc_reset_env(ipc_ctx* ctx, int env, const ipc_scene_desc* scene) {
  if (check_env(ctx, env) != IPC_OK || !scene) return IPC_EINVAL;
  std::shared_ptr<EnvLocal> L;
  std::string err;
  if (!build_env_local(*scene, env, ctx->prm, L, err)) {
    ctx->err = "ipc_reset_env: " + err;
    return IPC_EINVAL;
  }
  Pack& pk = ctx->pk;
  if (!same_topology(*pk.locals[env], *L)) {
    ctx->err = "ipc_reset_env: the scene's topology (mesh sizes, connectivity, pinned / attached / driven sets, "
               "bodies) differs from the env's";
    return IPC_EINVAL;
  }
  // the previous step may still read the tables
  CK(cudaStreamSynchronize(ctx->stream));
  patch_env_values(pk, env, *L);
  const EnvInfo& ev = pk.env[env];
  Dev& d = ctx->dev;
  cudaStream_t s = ctx->stream;
  auto up = [&](const void* dst, const void* src, size_t bytes) -> cudaError_t {
    return bytes ? cudaMemcpyAsync(const_cast<void*>(dst), src, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
  };
  const size_t r0 = ev.row_begin, R = ev.n_rows, t0 = ev.tet_begin, T = ev.n_tets, c0 = ev.cv_begin,
               NC = ev.n_cv, b0 = ev.body_begin, NB = ev.n_bodies, e0 = ev.edge_begin, NE = ev.n_edge,
               tr0 = ev.tri_begin, NT = ev.n_tri;
  CK(up(d.env_mu + env, &pk.env_mu[env], sizeof(double)));
  CK(up(d.env_lam + env, &pk.env_lam[env], sizeof(double)));
  CK(up(d.row_mass + r0, &pk.row_mass[r0], R * sizeof(double)));
  CK(up(d.row_xbar + 3 * r0, &pk.row_xbar[3 * r0], 3 * R * sizeof(double)));
  CK(up(d.Dm_inv + 9 * t0, &pk.Dm_inv[9 * t0], 9 * T * sizeof(double)));
  CK(up(d.tet_vol + t0, &pk.tet_vol[t0], T * sizeof(double)));
  if (NB) {
    CK(up(d.body_mass + b0, &pk.body_mass[b0], NB * sizeof(double)));
    CK(up(d.body_vol + b0, &pk.body_vol[b0], NB * sizeof(double)));
    CK(up(d.body_kappa + b0, &pk.body_kappa[b0], NB * sizeof(double)));
    CK(up(d.body_driven + b0, &pk.body_driven[b0], NB * sizeof(uint8_t)));
    CK(up(d.body_S + 9 * b0, &pk.body_S[9 * b0], 9 * NB * sizeof(double)));
  }
  CK(up(d.cv_xbar + 3 * c0, &pk.cv_xbar[3 * c0], 3 * NC * sizeof(double)));
  CK(up(d.cv_area + c0, &pk.cv_area[c0], NC * sizeof(double)));
  CK(up(d.cv_fixed + c0, &pk.cv_fixed[c0], NC * sizeof(uint8_t)));
  CK(up(d.edge_area + e0, &pk.edge_area[e0], NE * sizeof(double)));
  CK(up(d.edge_len2 + e0, &pk.edge_len2[e0], NE * sizeof(double)));
  CK(up(d.bv_perm[0] + c0, &pk.bv_perm[0][c0], NC * sizeof(int)));
  CK(up(d.bv_perm[1] + tr0, &pk.bv_perm[1][tr0], NT * sizeof(int)));
  CK(up(d.bv_perm[2] + e0, &pk.bv_perm[2][e0], NE * sizeof(int)));
  // rest state: x = targets = rest placement, velocities and multipliers zero
  CK(up(d.x + 3 * r0, &pk.rest_x[3 * r0], 3 * R * sizeof(double)));
  CK(up(d.s_tgt + 3 * r0, &pk.rest_x[3 * r0], 3 * R * sizeof(double)));
  CK(cudaMemsetAsync(d.v + 3 * r0, 0, 3 * R * sizeof(double), s));
  CK(cudaMemsetAsync(d.lam + 3 * r0, 0, 3 * R * sizeof(double), s));
  CK(cudaMemsetAsync(d.env_i + env * NUM_INTS + I_STATUS, 0, sizeof(int), s));
  CK(cudaStreamSynchronize(s));
  return IPC_OK;
}

ipc_status ipc_set_targets(ipc_ctx* ctx, int env, const double* y_target) {
  if (check_env(ctx, env) != IPC_OK || !y_target) return IPC_EINVAL;
  const EnvInfo& ev = ctx->pk.env[env];
  if (ev.n_bodies == 0) return IPC_OK;
  CK(cudaMemcpyAsync(ctx->dev.s_tgt + 3 * (size_t)(ev.row_begin + ev.gel_rows), y_target,
                     12 * sizeof(double) * ev.n_bodies, cudaMemcpyHostToDevice, ctx->stream));
  return IPC_OK;
}

ipc_status ipc_set_targets_all(ipc_ctx* ctx, const double* y_targets) {
  if (!ctx || !y_targets) return IPC_EINVAL;
  const size_t n = 12 * (size_t)ctx->max_bodies * ctx->pk.n_envs;
  if (n == 0) return IPC_OK;
  CK(cudaMemcpyAsync(ctx->dev.tgt_stage, y_targets, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  KL(ctx, KC_MISC, [&] { return launch_scatter_targets(ctx->dev, ctx->stream); });
  return last_cuda(ctx);
}

ipc_status ipc_set_targets_all_device(ipc_ctx* ctx, const double* dev_y_targets) {
  if (!ctx || !dev_y_targets) return IPC_EINVAL;
  const size_t n = 12 * (size_t)ctx->max_bodies * ctx->pk.n_envs;
  if (n == 0) return IPC_OK;
  CK(cudaMemcpyAsync(ctx->dev.tgt_stage, dev_y_targets, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  KL(ctx, KC_MISC, [&] { return launch_scatter_targets(ctx->dev, ctx->stream); });
  return last_cuda(ctx);
}

ipc_status ipc_step(ipc_ctx* ctx, const int32_t* env_ids, int n, int32_t* per_env_status, ipc_step_stats* stats) {
  if (!ctx) return IPC_EINVAL;
  ctx->step_t0 = std::chrono::steady_clock::now();
  std::vector<int> sel;
  if (!env_ids) {
    for (int e = 0; e < ctx->pk.n_envs; ++e) sel.push_back(e);
  } else {
    for (int i = 0; i < n; ++i) {
      if (check_env(ctx, env_ids[i]) != IPC_OK) return IPC_EINVAL;
      sel.push_back(env_ids[i]);
    }
  }
  ctx->last_sel = sel;
  if (sel.empty()) {  // nothing to step
    ctx->step_pending = false;
    if (stats) *stats = ipc_step_stats{};
    return IPC_OK;
  }
  const Dev& d = ctx->dev;
  cudaStream_t s = ctx->stream;
  ipc_status st;
  if (!env_ids) KL(ctx, KC_MISC, [&] { return launch_env_reset(d, 4, s); });  // every env
  else if ((st = select_envs(ctx, sel)) != IPC_OK) return st;
  if (ctx->graph_mode == 2 && !ctx->prof_on) {
    // the whole step as one graph: no host round trip until the results
    if (!ctx->step_exec && (st = capture_step(ctx)) != IPC_OK) return st;
    CK(cudaGraphLaunch(ctx->step_exec, s));
    ctx->step_graph_pending = true;
    ctx->step_pending = true;
    if ((st = last_cuda(ctx)) != IPC_OK) return st;
    if (!per_env_status && !stats) return IPC_OK;
    return ipc_step_results(ctx, per_env_status, stats);
  }
  KL(ctx, KC_MISC, [&] { return launch_env_reset(d, 0, s); });
  KL(ctx, KC_PREDICT, [&] { return launch_predict(d, I_SEL, s); });
  KL(ctx, KC_PREDICT, [&] { return launch_attach_targets(d, I_SEL, s); });
  const unsigned nmax = (unsigned)ctx->prm.newton_max;
  for (int it = 0; it < ctx->prm.newton_max; ++it) {
    if ((st = newton_iteration_host(ctx)) != IPC_OK) return st;
    // Newton iteration counter on the device
    KL(ctx, KC_MISC, [&] { return launch_flag_cond(d, s, I_ACTIVE, 2, 0, -1, -1, nmax, 0, 0); });
    if (count_flag(ctx, I_ACTIVE) == 0) break;
  }
  KL(ctx, KC_MISC, [&] { return launch_finalize(d, s); });
  if ((st = last_cuda(ctx)) != IPC_OK) return st;
  ctx->step_pending = true;
  return ipc_step_results(ctx, per_env_status, stats);
}

ipc_status ipc_step_results(ipc_ctx* ctx, int32_t* per_env_status, ipc_step_stats* stats) {
  if (!ctx) return IPC_EINVAL;
  if (!ctx->step_pending) {
    if (stats) *stats = ipc_step_stats{};
    return IPC_OK;
  }
  ipc_status st;
  if (ctx->step_graph_pending)
    CK(cudaMemcpyAsync(ctx->h_step_ctl, ctx->dev.step_ctl, 8 * sizeof(unsigned int), cudaMemcpyDeviceToHost,
                       ctx->stream));
  if ((st = sync_flags(ctx)) != IPC_OK) return st;
  if (ctx->step_graph_pending) {
    const ipc_ctx::StepLaunches& L = ctx->step_launches;
    const unsigned* c = ctx->h_step_ctl;
    ctx->launches += L.pre + (long long)c[0] * L.newton + (long long)c[4] * L.pcg_iter +
                     (long long)c[6] * L.ls_prep + (long long)c[5] * L.ls_trial + L.post;
    ctx->step_graph_pending = false;
    ctx->last_loop_iters = c[0];
    ctx->last_pcg_launches = c[4];
  } else {
    ctx->last_loop_iters = ctx->last_pcg_launches = 0;
  }
  ctx->step_pending = false;
  const std::vector<int>& sel = ctx->last_sel;
  ipc_step_stats S{};
  for (size_t i = 0; i < sel.size(); ++i) {
    const int* ei = ctx->h_int + sel[i] * NUM_INTS;
    if (per_env_status) per_env_status[i] = ei[I_STATUS];
    S.newton_iters = std::max(S.newton_iters, ei[I_NEWTON]);
    S.al_updates = std::max(S.al_updates, ei[I_AL]);
    S.pcg_iters += ei[I_PCGTOT];
    S.ls_trials += ei[I_LSTOT];
    S.max_pairs = std::max(S.max_pairs, ei[I_NPAIRS]);
    S.newton_env_iters += ei[I_NEWTON];
    S.al_env_updates += ei[I_AL];
    S.ccd_limited += ei[I_CCDCUT];
    S.accd_iters += ei[I_ACCDIT];
    S.accd_iters_max = std::max(S.accd_iters_max, ei[I_ACCDMAX]);
    S.alpha_sum += ctx->h_dbl[sel[i] * NUM_SCALARS + S_ASUM];
    S.act_pair_iters += (long long)ctx->h_dbl[sel[i] * NUM_SCALARS + S_APCG];
    S.pair_evals += ei[I_PAIRTOT];
    S.swept_pairs += ei[I_SWEPTTOT];
  }
  S.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - ctx->step_t0).count();
  S.loop_iters = ctx->last_loop_iters;
  S.pcg_launches = ctx->last_pcg_launches;
  if (stats) *stats = S;
  return IPC_OK;
}

ipc_status ipc_rollout(ipc_ctx* ctx, const int32_t* env_ids, int n, int n_steps, const int32_t* steps_per_env,
                       const double* dev_targets, int32_t* per_env_status, int32_t* per_env_steps,
                       ipc_step_stats* stats) {
  if (!ctx || n_steps < 0 || (n_steps > 0 && !dev_targets && ctx->max_bodies > 0)) return IPC_EINVAL;
  ctx->step_t0 = std::chrono::steady_clock::now();
  std::vector<int> sel;
  if (!env_ids) {
    for (int e = 0; e < ctx->pk.n_envs; ++e) sel.push_back(e);
  } else {
    for (int i = 0; i < n; ++i) {
      if (check_env(ctx, env_ids[i]) != IPC_OK) return IPC_EINVAL;
      sel.push_back(env_ids[i]);
    }
  }
  ctx->last_sel = sel;
  const Dev& d = ctx->dev;
  cudaStream_t s = ctx->stream;
  ipc_status st;
  if (!env_ids) KL(ctx, KC_MISC, [&] { return launch_env_reset(d, 4, s); });
  else if ((st = select_envs(ctx, sel)) != IPC_OK) return st;
  {
    // per-env step limits (I_RLIMIT column): n_steps, or the caller's
    std::vector<int> col(ctx->pk.n_envs, n_steps);
    for (size_t i = 0; i < sel.size(); ++i)
      if (steps_per_env) {
        if (steps_per_env[i] < 0) return IPC_EINVAL;
        col[sel[i]] = std::min(steps_per_env[i], n_steps);
      }
    CK(cudaMemcpy2DAsync(ctx->dev.env_i + I_RLIMIT, NUM_INTS * sizeof(int), col.data(), sizeof(int), sizeof(int),
                         ctx->pk.n_envs, cudaMemcpyHostToDevice, s));  // pageable: staged before return
  }
  // every env's step ends within newton_max Newton iterations, each within
  // ceil(pcg_max / window) + 1 loop iterations: the cap only guards
  const unsigned long long w = ctx->prm.rollout_pcg_window > 0 ? (unsigned long long)ctx->prm.rollout_pcg_window
                                                               : (unsigned long long)ctx->prm.pcg_max;
  const unsigned long long per_newton = ((unsigned long long)ctx->prm.pcg_max + w - 1) / w + 1;
  const unsigned long long cap =
      (unsigned long long)n_steps * ((unsigned long long)ctx->prm.newton_max + 1) * per_newton + 2;
  KL(ctx, KC_MISC, [&] { return launch_roll_setup(d, dev_targets, n_steps, cap, s); });
  if (!ctx->prof_on) {
    if (!ctx->roll_exec && (st = capture_roll(ctx)) != IPC_OK) return st;
    CK(cudaGraphLaunch(ctx->roll_exec, s));
    CK(cudaMemcpyAsync(ctx->h_step_ctl, ctx->dev.step_ctl, 8 * sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    ctx->roll_pending = true;
    if ((st = last_cuda(ctx)) != IPC_OK) return st;
  } else {
    // the same loop driven from the host with plain launches (per-kernel
    // timing needs them)
    KL(ctx, KC_MISC, [&] { return launch_roll_init(d, s); });
    if ((st = sync_flags(ctx)) != IPC_OK) return st;
    for (unsigned long long it = 0; it < cap && count_flag(ctx, I_LIVE) > 0; ++it) {
      KL(ctx, KC_PREDICT, [&] { return launch_roll_begin(d, s); });
      if ((st = newton_iteration_host(ctx)) != IPC_OK) return st;
      KL(ctx, KC_MISC, [&] { return launch_roll_end(d, s); });
      if ((st = sync_flags(ctx)) != IPC_OK) return st;
    }
    ctx->roll_pending = true;
  }
  ctx->step_pending = false;
  if (!per_env_status && !per_env_steps && !stats) return IPC_OK;
  return ipc_rollout_results(ctx, per_env_status, per_env_steps, stats);
}

ipc_status ipc_rollout_results(ipc_ctx* ctx, int32_t* per_env_status, int32_t* per_env_steps,
                               ipc_step_stats* stats) {
  if (!ctx) return IPC_EINVAL;
  if (!ctx->roll_pending) {
    if (stats) *stats = ipc_step_stats{};
    return IPC_OK;
  }
  ipc_status st;
  if ((st = sync_flags(ctx)) != IPC_OK) return st;
  if (!ctx->prof_on) {
    const ipc_ctx::RollLaunches& L = ctx->roll_launches;
    const unsigned* c = ctx->h_step_ctl;
    // c[0] counts the loop's condition evaluations (one before the loop)
    const long long iters = c[0] > 0 ? (long long)c[0] - 1 : 0;
    ctx->launches += L.pre + iters * L.iter + (long long)c[4] * L.pcg_iter + (long long)c[6] * L.ls_prep +
                     (long long)c[5] * L.ls_trial;
    ctx->last_loop_iters = iters;
    ctx->last_pcg_launches = c[4];
  } else {
    ctx->last_loop_iters = ctx->last_pcg_launches = 0;
  }
  ctx->roll_pending = false;
  const std::vector<int>& sel = ctx->last_sel;
  ipc_step_stats S{};
  for (size_t i = 0; i < sel.size(); ++i) {
    const int* ei = ctx->h_int + sel[i] * NUM_INTS;
    if (per_env_status) per_env_status[i] = ei[I_STATUS];
    if (per_env_steps) per_env_steps[i] = ei[I_RSTEP];
    S.newton_iters = std::max(S.newton_iters, ei[I_RNEWTONMAX]);
    S.al_updates = std::max(S.al_updates, ei[I_RAL]);
    S.pcg_iters += ei[I_RPCG];
    S.ls_trials += ei[I_RLS];
    S.max_pairs = std::max(S.max_pairs, ei[I_RPAIRSMAX]);
    S.newton_env_iters += ei[I_RNEWTON];
    S.al_env_updates += ei[I_RAL];
    S.ccd_limited += ei[I_RCCDCUT];
    S.accd_iters += ei[I_RACCDIT];
    S.accd_iters_max = std::max(S.accd_iters_max, ei[I_RACCDMAX]);
    S.alpha_sum += ctx->h_dbl[sel[i] * NUM_SCALARS + S_RASUM];
    S.act_pair_iters += (long long)ctx->h_dbl[sel[i] * NUM_SCALARS + S_RAPCG];
    S.pair_evals += ei[I_RPAIR];
    S.swept_pairs += ei[I_RSWEPT];
  }
  S.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - ctx->step_t0).count();
  S.loop_iters = ctx->last_loop_iters;
  S.pcg_launches = ctx->last_pcg_launches;
  if (stats) *stats = S;
  return IPC_OK;
}

ipc_status ipc_env_stats(const ipc_ctx* ctx, int env, int32_t* out) {
  if (check_env(ctx, env) != IPC_OK || !out) return IPC_EINVAL;
  const int* ei = ctx->h_int + env * NUM_INTS;
  const int k[IPC_ENV_STATS] = {I_STATUS, I_NEWTON, I_AL,      I_PCGTOT,  I_LSTOT,   I_CCDCUT,
                                I_ACCDMAX, I_NPAIRS, I_ACCDIT, I_PAIRTOT, I_SWEPTTOT};
  for (int i = 0; i < IPC_ENV_STATS; ++i) out[i] = ei[k[i]];
  return IPC_OK;
}

ipc_status ipc_read_gel_surface(ipc_ctx* ctx, int env, double* out_xyz, int capacity, int* n_written) {
  if (check_env(ctx, env) != IPC_OK) return IPC_EINVAL;
  const EnvInfo& ev = ctx->pk.env[env];
  std::vector<double> rows;
  ipc_status st = download_rows(ctx, env, ctx->dev.x, rows);
  if (st != IPC_OK) return st;
  // coated rows are listed in increasing user id order
  int n = ev.n_coated;
  for (int i = 0; i < std::min(n, capacity); ++i) {
    int r = ctx->pk.coated_row[ev.coated_begin + i] - ev.row_begin;
    for (int c = 0; c < 3; ++c) out_xyz[3 * i + c] = rows[3 * r + c];
  }
  if (n_written) *n_written = n;
  return IPC_OK;
}

ipc_status ipc_read_gel_surface_all(ipc_ctx* ctx, double* out_xyz, size_t capacity_rows, size_t* rows_written) {
  if (!ctx || !out_xyz) return IPC_EINVAL;
  size_t n = std::min<size_t>(capacity_rows, ctx->pk.n_coated);
  KL(ctx, KC_MISC, [&] { return launch_gather_coated(ctx->dev, ctx->stream); });
  if (n) CK(cudaMemcpyAsync(out_xyz, ctx->dev.out_stage, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (rows_written) *rows_written = ctx->pk.n_coated;
  return last_cuda(ctx);
}

// ---------------------------------------------------------------- diagnostics
ipc_status ipc_debug_eval(ipc_ctx* ctx, int env, double* energy, double* grad, const double* vec, double* hvec) {
  if (check_env(ctx, env) != IPC_OK) return IPC_EINVAL;
  const EnvInfo& ev = ctx->pk.env[env];
  const Dev& d = ctx->dev;
  ipc_status st;
  if ((st = begin_single(ctx, env)) != IPC_OK) return st;
  if ((st = assemble_system(ctx, ctx->stream)) != IPC_OK) return st;
  std::vector<double> rows;
  if (grad) {
    if ((st = download_rows(ctx, env, d.g, rows)) != IPC_OK) return st;
    rows_to_dof(ctx, env, rows, grad);
  }
  if (energy) {
    if ((st = select_envs(ctx, {env}, I_LS)) != IPC_OK) return st;
    CK(cudaMemsetAsync(d.p, 0, 3 * sizeof(double) * d.n_rows, ctx->stream));
    KL(ctx, KC_CVPOS, [&] { return launch_cv_pos(d, I_LS, true, ctx->stream); });
    KL(ctx, KC_ENERGY, [&] { return launch_energy(d, 0, 0, ctx->stream); });
    if ((st = select_envs(ctx, {}, I_LS)) != IPC_OK) return st;
    if ((st = sync_flags(ctx)) != IPC_OK) return st;
    *energy = ctx->h_dbl[env * NUM_SCALARS + S_E0];
  }
  if (vec && hvec) {
    std::vector<double> vr;
    dof_to_rows(ctx, env, vec, vr);
    // the mat-vec reads the PCG direction (FP32 rows in mixed mode): loaded
    // from FP64 rows staged in d.z
    if ((st = upload_rows(ctx, env, d.z, vr)) != IPC_OK) return st;
    if ((st = select_envs(ctx, {env}, I_PCG)) != IPC_OK) return st;
    // one mat-vec with z = v, beta = 0 and d_{-1} = 0 (so d_0 = v)
    KL(ctx, KC_MISC, [&] { return launch_debug_dir_from_rows(d, ctx->stream); });
    KL(ctx, KC_PCGINIT, [&] { return launch_pcg_begin(d, ctx->stream, 0, 0); });
    KL(ctx, KC_SPMV, [&] { return launch_pcg_matvec(d, ctx->stream); });
    KL(ctx, KC_PAIRSPMV, [&] { return launch_pcg_pairs(d, ctx->stream); });
    KL(ctx, KC_FRICSPMV, [&] { return launch_fric_spmv(d, ctx->stream); });
    KL(ctx, KC_MISC, [&] { return launch_debug_q_to_rows(d, ctx->stream); });
    if ((st = select_envs(ctx, {}, I_PCG)) != IPC_OK) return st;
    if ((st = last_cuda(ctx)) != IPC_OK) return st;
    if ((st = download_rows(ctx, env, d.q, rows)) != IPC_OK) return st;
    rows_to_dof(ctx, env, rows, hvec);
  }
  return IPC_OK;
}

ipc_status ipc_debug_newton_dir(ipc_ctx* ctx, int env, double* p, int* pcg_iters) {
  if (check_env(ctx, env) != IPC_OK || !p) return IPC_EINVAL;
  ipc_status st;
  if ((st = begin_single(ctx, env)) != IPC_OK) return st;
  if ((st = assemble_system(ctx, ctx->stream)) != IPC_OK) return st;
  if ((st = run_pcg(ctx)) != IPC_OK) return st;
  if ((st = sync_flags(ctx)) != IPC_OK) return st;
  if (pcg_iters) *pcg_iters = ctx->h_int[env * NUM_INTS + I_PCGIT];
  std::vector<double> rows;
  if ((st = download_rows(ctx, env, ctx->dev.p, rows)) != IPC_OK) return st;
  rows_to_dof(ctx, env, rows, p);
  return IPC_OK;
}

ipc_status ipc_debug_pcg_wait_out(ipc_ctx* ctx, int env, int* env_status, float* ms) {
  if (check_env(ctx, env) != IPC_OK) return IPC_EINVAL;
  const Dev& d = ctx->dev;
  cudaStream_t s = ctx->stream;
  if (pcg_iters_per_launch(d, 0xffffffffu) <= 1) {
    ctx->err = "pcg_wait_out: needs the multi-iteration PCG kernel (pcg_fused > 0, pcg_iters_per_launch > 1)";
    return IPC_EINVAL;
  }
  ipc_status st;
  if ((st = begin_single(ctx, env)) != IPC_OK) return st;
  if ((st = assemble_system(ctx, s)) != IPC_OK) return st;
  KL(ctx, KC_PCGINIT, [&] { return launch_pcg_init(d, s); });
  KL(ctx, KC_PCGINIT, [&] { return launch_pcg_begin(d, s, 0, 0); });
  // the env's first products wait for an update round that never completes
  KL(ctx, KC_MISC, [&] { return launch_debug_set_updk(d, env, -1, s); });
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  CK(cudaEventRecord(a, s));
  pcg_iteration(ctx, s);
  CK(cudaEventRecord(b, s));
  CK(cudaEventSynchronize(b));
  float t = 0.f;
  CK(cudaEventElapsedTime(&t, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if ((st = last_cuda(ctx)) != IPC_OK) return st;
  if ((st = sync_flags(ctx)) != IPC_OK) return st;
  if (env_status) *env_status = ctx->h_int[env * NUM_INTS + I_STATUS];
  if (ms) *ms = t;
  return IPC_OK;
}

ipc_status ipc_debug_pairs(ipc_ctx* ctx, int env, const double* cv_x, const double* cv_x_end, int32_t* out,
                           int capacity, int* n_pairs) {
  if (check_env(ctx, env) != IPC_OK || !cv_x) return IPC_EINVAL;
  const Pack& pk = ctx->pk;
  const EnvInfo& ev = pk.env[env];
  const Dev& d = ctx->dev;
  ipc_status st;
  // contact vertex positions (internal order) from caller ids
  std::vector<double> X(3 * (size_t)ev.n_cv), P(3 * (size_t)ev.n_cv, 0.0);
  for (int i = 0; i < ev.n_cv; ++i) {
    int u = pk.cv_uid[ev.cv_begin + i];
    for (int c = 0; c < 3; ++c) {
      X[3 * i + c] = cv_x[3 * u + c];
      if (cv_x_end) P[3 * i + c] = cv_x_end[3 * u + c] - cv_x[3 * u + c];
    }
  }
  CK(cudaMemcpyAsync(d.cvx + 3 * (size_t)ev.cv_begin, X.data(), X.size() * sizeof(double), cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaMemcpyAsync(d.cvp + 3 * (size_t)ev.cv_begin, P.data(), P.size() * sizeof(double), cudaMemcpyHostToDevice,
                     ctx->stream));
  if ((st = select_envs(ctx, {env})) != IPC_OK) return st;
  KL(ctx, KC_OBJBOX, [&] { return launch_obj_box(d, I_SEL, cv_x_end != nullptr, ctx->stream); });
  KL(ctx, KC_MISC, [&] { return launch_env_reset(d, 6, ctx->stream); });
  KL(ctx, KC_BROAD, [&] { return launch_broad(d, I_SEL, cv_x_end != nullptr, ctx->stream); });
  if ((st = last_cuda(ctx)) != IPC_OK) return st;
  if ((st = sync_flags(ctx)) != IPC_OK) return st;
  int n = ctx->h_int[env * NUM_INTS + I_NPAIRS];
  if (n_pairs) *n_pairs = n;
  int m = std::min(n, ev.pair_cap);
  std::vector<int4> v(m);
  std::vector<int> kind(m);
  if (m) {
    CK(cudaMemcpyAsync(v.data(), d.pair_v + ev.pair_begin, m * sizeof(int4), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(kind.data(), d.pair_kind + ev.pair_begin, m * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  for (int i = 0; i < std::min(m, capacity); ++i) {
    out[5 * i] = kind[i];
    out[5 * i + 1] = pk.cv_uid[v[i].x];
    out[5 * i + 2] = pk.cv_uid[v[i].y];
    out[5 * i + 3] = pk.cv_uid[v[i].z];
    out[5 * i + 4] = pk.cv_uid[v[i].w];
  }
  return n > ev.pair_cap ? IPC_EOVERFLOW : IPC_OK;
}

ipc_status ipc_debug_accd(ipc_ctx* ctx, int env, const double* dir, double* alpha) {
  if (check_env(ctx, env) != IPC_OK || !dir || !alpha) return IPC_EINVAL;
  const Dev& d = ctx->dev;
  ipc_status st;
  std::vector<double> rows;
  dof_to_rows(ctx, env, dir, rows);
  if ((st = upload_rows(ctx, env, d.p, rows)) != IPC_OK) return st;
  if ((st = select_envs(ctx, {env}, I_LS)) != IPC_OK) return st;
  KL(ctx, KC_CVPOS, [&] { return launch_cv_pos(d, I_LS, true, ctx->stream); });
  KL(ctx, KC_OBJBOX, [&] { return launch_obj_box(d, I_LS, true, ctx->stream); });
  KL(ctx, KC_MISC, [&] { return launch_env_reset(d, 5, ctx->stream); });
  KL(ctx, KC_BROAD, [&] { return launch_broad(d, I_LS, true, ctx->stream); });
  // S_ACCD = 1 then min over pairs
  std::vector<double> one(1, 1.0);
  CK(cudaMemcpyAsync(d.env_s + env * NUM_SCALARS + S_ACCD, one.data(), sizeof(double), cudaMemcpyHostToDevice,
                     ctx->stream));
  KL(ctx, KC_ACCD, [&] { return launch_accd(d, ctx->stream); });
  if ((st = select_envs(ctx, {}, I_LS)) != IPC_OK) return st;
  if ((st = last_cuda(ctx)) != IPC_OK) return st;
  if ((st = sync_flags(ctx)) != IPC_OK) return st;
  *alpha = ctx->h_dbl[env * NUM_SCALARS + S_ACCD];
  return IPC_OK;
}

ipc_status ipc_profile_enable(ipc_ctx* ctx, int on) {
  if (!ctx) return IPC_EINVAL;
  if (ctx->prof_launches.empty()) {
    ctx->prof_launches.assign(KC_COUNT, 0);
    ctx->prof_ms.assign(KC_COUNT, 0.0);
  }
  ctx->prof_on = on != 0;
  return IPC_OK;
}

ipc_status ipc_profile_reset(ipc_ctx* ctx) {
  if (!ctx) return IPC_EINVAL;
  cudaStreamSynchronize(ctx->stream);
  prof_flush(ctx);
  ctx->prof_launches.assign(KC_COUNT, 0);
  ctx->prof_ms.assign(KC_COUNT, 0.0);
  return IPC_OK;
}

int ipc_profile_count(const ipc_ctx* ctx) { return ctx ? (int)KC_COUNT : 0; }

ipc_status ipc_profile_get(const ipc_ctx* ctx, int i, const char** name, long long* launches, double* ms) {
  if (!ctx || i < 0 || i >= KC_COUNT) return IPC_EINVAL;
  if (name) *name = KC_NAME[i];
  if (launches) *launches = ctx->prof_launches.empty() ? 0 : ctx->prof_launches[i];
  if (ms) *ms = ctx->prof_ms.empty() ? 0.0 : ctx->prof_ms[i];
  return IPC_OK;
}

long long ipc_launch_count(const ipc_ctx* ctx) { return ctx ? ctx->launches : 0; }

ipc_status ipc_system_sizes(const ipc_ctx* ctx, int env, long long* real_blocks, long long* stored_blocks, int* rows,
                            int* tets) {
  if (check_env(ctx, env) != IPC_OK) return IPC_EINVAL;
  const Pack& pk = ctx->pk;
  const EnvInfo& ev = pk.env[env];
  long long stored = 0, real = 0;
  for (int ch = ev.chunk_begin; ch < ev.chunk_begin + ev.n_chunks; ++ch) {
    stored += 32LL * pk.chunk_slots[ch];
    for (int sl = 0; sl < pk.chunk_slots[ch]; ++sl)
      for (int l = 0; l < 32; ++l) {
        long long blk = pk.chunk_ptr[ch] + 32LL * sl + l;
        int r = ch * 32 + l;  // global row
        int lr = r - ev.row_begin;
        bool gel = lr < ev.n_verts;
        bool body = lr >= ev.gel_rows && lr < ev.gel_rows + 4 * ev.n_bodies;
        if (gel && (sl == 0 || pk.sell_col[blk] != r)) ++real;
        if (body && sl < 4) ++real;
      }
  }
  if (real_blocks) *real_blocks = real;
  if (stored_blocks) *stored_blocks = stored;
  if (rows) *rows = ev.n_rows;
  if (tets) *tets = ev.n_tets;
  return IPC_OK;
}

// ---------------------------------------------------------------- element kernels
ipc_status ipc_k_tet(int n, const double* x, const double* Dm_inv, const double* vol, double mu, double lam,
                     double* energy, double* grad, double* hess, int project, void* stream) {
  if (n < 0 || (n > 0 && (!x || !Dm_inv || !vol)) || project < 0 || project > 2) return IPC_EINVAL;
  launch_k_tet(n, x, Dm_inv, vol, mu, lam, energy, grad, hess, project, reinterpret_cast<cudaStream_t>(stream));
  return cudaGetLastError() == cudaSuccess ? IPC_OK : IPC_ECUDA;
}

ipc_status ipc_k_barrier(int n, const double* X, const int32_t* is_ee, const double* weight, const double* eps_x,
                         double dhat, double* energy, double* grad, double* hess, int project, void* stream) {
  if (n < 0 || (n > 0 && (!X || !is_ee || !weight)) || !(dhat > 0) || project < 0 || (project & ~8) > 2)
    return IPC_EINVAL;
  launch_k_barrier(n, X, is_ee, weight, eps_x, dhat, energy, grad, hess, project,
                   reinterpret_cast<cudaStream_t>(stream));
  return cudaGetLastError() == cudaSuccess ? IPC_OK : IPC_ECUDA;
}

ipc_status ipc_k_accd(int n, const double* X0, const double* P, const int32_t* is_ee, double s, int max_iter,
                      double* toi, int32_t* iters, void* stream) {
  if (n < 0 || (n > 0 && (!X0 || !P || !is_ee || !toi)) || !(s > 0 && s < 1) || max_iter < 1) return IPC_EINVAL;
  launch_k_accd(n, X0, P, is_ee, s, max_iter, toi, iters, reinterpret_cast<cudaStream_t>(stream));
  return cudaGetLastError() == cudaSuccess ? IPC_OK : IPC_ECUDA;
}

}  // extern "C"
