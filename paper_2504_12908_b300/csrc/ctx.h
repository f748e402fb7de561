// Device context: every array the kernels touch, carved out of the caller's
// workspace.  `Dev` is passed by value to kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <chrono>
#include <string>
#include <vector>

#include "scene.h"

namespace ipc {

// per-env double scalars
enum EnvScalar {
  S_RZ = 0,     // PCG r.z
  S_DQ,         // PCG d.q
  S_RR,         // PCG r.r
  S_RR0,        // PCG |b|^2
  S_PALPHA,     // PCG alpha
  S_PBETA,      // PCG beta
  S_PNORM,      // Newton |p|_inf (full space)
  S_CRES,       // AL constraint residual |q - s|_inf (full space)
  S_ACCD,       // CCD step bound
  S_ALPHA,      // line-search step
  S_E0,         // energy at the line-search start
  S_E1,         // energy at the trial step
  S_MIND,       // min pair distance (diagnostics)
  S_ASUM,       // accepted line-search steps this step, summed
  S_DQC,        // PCG d.q, contact part (pair and friction terms, summed by atomics)
  S_RASUM,      // rollout: S_ASUM summed over the env's steps
  S_APCG,       // active contact pairs x PCG iterations, summed over this step's solves
  S_RAPCG,      // rollout: S_APCG summed over the env's steps
  NUM_SCALARS
};

// per-env int state
enum EnvInt {
  I_ACTIVE = 0,   // still iterating Newton in this step
  I_PCG,          // PCG still running
  I_LS,           // line search still running
  I_STATUS,       // ipc_status of this env for the current step
  I_NEWTON,       // Newton iterations done
  I_AL,           // AL updates done
  I_LSIT,         // halvings in the current line search
  I_PCGIT,        // PCG iterations in the current solve
  I_MODE,         // after the Newton check: 0 line search, 1 converged, 2 AL update
  I_NPAIRS,       // candidate pairs in the current list
  I_OVERFLOW,     // pair list overflowed
  I_ACCEPT,       // line search accepted this trial
  I_PCGTOT,       // PCG iterations this step
  I_LSTOT,        // line-search trials this step
  I_SEL,          // selected for this ipc_step call
  I_FLAG,         // scratch flag (inverted tet found)
  I_CCDCUT,       // line searches starting below alpha = 1 this step
  I_ACCDIT,       // ACCD advancement iterations this step (all pairs)
  I_ACCDMAX,      // most ACCD iterations one pair took this step
  I_NFRIC,        // lagged friction records of this step
  I_NACT,         // active contact pairs (d < dhat) of this Newton iteration
  I_GEN,          // Newton iterations ever run (tags the rows contact terms touch)
  I_PAIRTOT,      // static candidate pairs evaluated this step (all Newton iterations)
  I_SWEPTTOT,     // swept candidate pairs of this step's line searches
  I_NEWT,         // starts a Newton iteration now (in the step, no solve carried over, no decision pending)
  I_DEC,          // its PCG solve ended: the Newton decision is pending
  I_PHASE,        // fused PCG iteration: the env's pair and mat-vec items finished
  I_LISTROW,      // index of the env's first row item in the PCG work list
  I_UPDK,         // multi-iteration PCG kernel: the env's iterations completed in the launch
  // rollout (ipc_rollout: each env runs its own sequence of steps)
  I_RSTEP,        // steps completed in this rollout
  I_BEGIN,        // begins its next step at the top of the next loop iteration
  I_RUN,          // inside a step
  I_ENDNOW,       // its step ended in this loop iteration
  I_LIVE,         // running a step or about to begin one
  I_RLIMIT,       // steps this env runs in the rollout (at most the call's n_steps)
  I_RNEWTON,      // the per-step counters above, summed (max for *MAX) over the rollout
  I_RNEWTONMAX,
  I_RAL,
  I_RPCG,
  I_RLS,
  I_RCCDCUT,
  I_RACCDIT,
  I_RACCDMAX,
  I_RPAIR,
  I_RSWEPT,
  I_RPAIRSMAX,
  NUM_INTS
};

struct Dev {
  int n_envs, n_rows, n_tets, n_cv, n_tri, n_edge, n_obj, n_bodies, n_chunks, n_coated;
  long long n_blocks, n_pairs_cap;
  // parameters
  double h, grav[3], dhat, kappa, newton_tol, pcg_tol, accd_s, al_kappa, ee_moll;
  int newton_max, pcg_max, ls_max, accd_max, al_max;
  int abs_after;                // Newton iterations per step that clamp negative eigenvalues;
                                // later iterations use their absolute values
  int prec;                     // 0 FP64, 1 mixed (FP32 Hessians and mat-vec)
  // launch shapes (ipc_autotune): SpMV slots in flight per lane (2, 4, 8;
  // 0 = the default, 2)
  int spmv_unroll;
  double fr_mu, fr_eh;          // friction coefficient; eps_v * h (fr_mu = 0: no friction)
  // static tables
  const int *env_row_off, *env_tet_off, *env_cv_off, *env_tri_off, *env_edge_off, *env_obj_off,
      *env_body_off, *env_chunk_off, *env_coated_off, *env_pair_cap, *env_pair_off;
  const double *env_mu, *env_lam;
  const int* cta_env;
  const int* env_has_driven;    // env has driven bodies or attached gel rows
  const double* row_mass;
  const uint8_t* row_kind;
  const int* row_body;
  const double* row_xbar;
  const int *vt_ptr, *vt_src;
  const int* tets;
  const double *Dm_inv, *tet_vol;
  const int* chunk_slots;
  const long long* chunk_ptr;
  const int *sell_col, *asm_ptr, *asm_src;
  const int *body_row, *body_env, *body_cv_begin, *body_nv;
  const double *body_mass, *body_S, *body_vol, *body_kappa;
  const uint8_t* body_driven;
  const int *cv_row, *cv_body, *cv_obj, *cv_uid;
  const double *cv_xbar, *cv_area;
  const uint8_t* cv_fixed;
  const int *tri, *tri_obj, *edge, *edge_obj;
  const double *edge_area, *edge_len2;
  const int *obj_env, *obj_local, *obj_cv_begin, *obj_cv_end, *obj_tri_begin, *obj_tri_end,
      *obj_edge_begin, *obj_edge_end, *obj_size;
  const unsigned long long* obj_exclude;
  const int* coated_row;
  // broad-phase hierarchy per primitive kind (0 points, 1 triangles, 2
  // edges): Morton-ordered primitives of each object in clusters of 32 and
  // superclusters of 32 clusters, boxes refitted at every candidate search
  const int *bv_perm[3], *bv_cl_obj[3], *bv_sc_obj[3], *obj_cl_begin[3], *obj_sc_begin[3];
  int bv_n_cl[3], bv_n_sc[3];
  double *bv_cl_box[3], *bv_sc_box[3];
  // state and work (row space: 3 doubles per row)
  double *x, *v, *xn, *xt, *s_tgt, *lam;
  double *p, *g, *r, *z, *d, *q, *qc;
  float4 *z4, *d4, *q4;         // mixed mode: the PCG vectors z, d, q as FP32 rows (16 B)
  // The PCG direction is double-buffered: iteration k reads d_{k-1} from one
  // buffer and writes d_k = z_k + beta d_{k-1} into the other (d / d4 when
  // k is even, db / d4b when odd).
  double* db;
  float4* d4b;
  uint8_t* row_touch;           // per row: 1 + (I_GEN % 255) of the Newton iteration whose
                                // contact terms write the row's contact accumulator qc
  // device-side PCG work list (rebuilt on the device when an env stops):
  int* pcg_list;                // [n_envs] envs still in PCG
  int* pcg_pair_off;            // [n_envs + 1] prefix of their groups of 8 active pairs
  int* pcg_row_off;             // [n_envs + 1] prefix of their 128-row CTAs
  int2* pcg_item;               // per row item: (env, global row CTA)
  int2* pcg_pitem;              // per pair item: (env, group of 8 active pairs)
  int2* pcg_fitem;              // per friction item: (env, group of 128 friction records)
  int* pcg_fric_off;            // [n_envs + 1] prefix of the listed envs' friction items
  unsigned int* pcg_ctl;        // [0] CTAs arrived in the update kernel, [1] PCG iteration,
                                // [2] envs in the list, [3] items of stopped envs, [4] envs
                                // solving, [5..10] the fused kernels' counters (PcgCtl)
  int* pcg_ritem;               // fused kernel: update items in the order their envs became
                                // ready (-1: slot not written)
  int pcg_grid;                 // CTAs of the persistent PCG row kernels
  int pcg_fused;                // 1 / 2: a PCG iteration is one kernel (k_pcg_iter; update items in
                                // ready order / env order) when friction is off; 0: three kernels
  int pcg_grid_fused;           // CTAs of k_pcg_iter (its resident CTAs)
  int pcg_iter_bound;           // k_pcg_iter's register bound: 1 on (default), 0 off (ipc_autotune)
  int pcg_multi;                // PCG iterations per launch of the fused kernel (> 1: k_pcg_multi)
  int pcg_grid_multi;           // CTAs of k_pcg_multi (its resident CTAs)
  int asm_block;                // threads per CTA of the gather assembly (ipc_autotune)
  int pairs_grid;               // CTAs of the candidate-pair search (ipc_autotune)
  int pcg_grid_pairs;           // CTAs of the persistent contact mat-vec
  unsigned long long* roll_ctl; // rollout: [0] address of the target table, [1] steps, [2] loop cap
  unsigned long long* check_word;  // bounds-checked builds: [0] first violation's code, [1] its index
  unsigned int* step_ctl;       // per step (device-side loops): [0] Newton iterations done,
                                // [1] trials of the current line search, [2] envs still in
                                // Newton, [3] envs in a line search, [4] PCG iterations,
                                // [5] line-search trials, [6] line searches
  void* pc;                     // 6 per row: symmetric inverse of the diagonal block
                                // (double, or float in mixed mode)
  double* pc_acc;               // 9 per row
  double *body_pc, *body_pc_acc, *body_g, *body_H, *body_E;  // per body 144 / 144 / 12 / 144 / 1
  void* sell_val;               // n_blocks * 9 (double, or float in mixed mode)
  double *tetG, *tetE;          // 12 / 1 per tet
  void* tetH;                   // 144 per tet (double, or float in mixed mode)
  double* row_E;
  double *cvx, *cvp;            // 3 per contact vertex
  double* obj_box;              // 6 per object
  double *cv_box, *tri_box, *edge_box;  // 6 per primitive
  int4* bp_items;               // broad-phase worklist (kind, query, object, env)
  int* bp_count;
  int* bp_overflow;
  int bp_cap;
  int4* pair_v;                 // contact vertex ids
  int* pair_kind;               // 0 PT, 1 EE
  double *pair_w, *pair_eps, *pair_E;
  void* pair_H;                 // 78 per active pair, by its slot s: entry j of the packed upper
                                // triangle at ((s / 32) * 78 + j) * 32 + s % 32 (double, or float in mixed mode)
  uint8_t* pair_act;
  int* pair_scan;                // n_envs + 1: exclusive scan of pair counts
  int4* act_v;                   // contact points of each active (d < dhat) pair, by slot: the
                                 // env's active pairs fill slots env_pair_off[e] + [0, I_NACT)
  // lagged friction records (segments like the pair list, I_NFRIC per env)
  int4* fr_v;                    // contact points of the pair
  double *fr_w, *fr_T, *fr_rn;   // closest-point weights (4), tangent basis (6), r at x^n (3)
  double *fr_ml, *fr_S, *fr_E;   // mu lambda; h^2 T M T^T (6, symmetric); energy
  int* fr_scan;                  // n_envs + 1: exclusive scan of the active envs' record counts
                                 // (rebuilt every Newton iteration)
  int4* accd_tail;               // ACCD pairs left for the warp-parallel phase: (slot, env, iterations, -)
  double* accd_tail_t;           // their certified time so far
  unsigned int* accd_tail_ctl;   // [entries, finished CTAs]; zero between launches
  double* cta_part;             // 4 per row CTA
  unsigned int* env_cnt;        // last-CTA counters (2 per env)
  double* tgt_stage;            // [n_envs][max_bodies][12] host targets
  double* out_stage;            // [n_coated][3] coated-surface positions
  int max_bodies;
  double* env_s;                // NUM_SCALARS per env
  int* env_i;                   // NUM_INTS per env
};

struct Layout {
  size_t total = 0;
  std::vector<std::pair<void**, size_t>> items;  // (slot, bytes)
};

}  // namespace ipc

struct ipc_ctx {
  ipc::Pack pk;
  ipc::Dev dev;
  ipc_params prm;
  cudaStream_t stream = nullptr;
  int device = -1;            // CUDA device of the stream / workspace (set at create)
  char* ws = nullptr;
  size_t ws_bytes = 0;
  std::string err;
  int* h_int = nullptr;       // pinned read-back (NUM_INTS * n_envs ints)
  unsigned int* h_ctl = nullptr;  // pinned read-back of Dev::pcg_ctl (8)
  double* h_dbl = nullptr;    // pinned read-back (NUM_SCALARS * n_envs doubles)
  int max_bodies = 0;
  std::vector<int> n_cta_env;  // row CTAs per env
  // Two high-priority side streams for the small, latency-bound launches
  // that are independent of the element kernels (per-pair barrier terms and
  // per-body ABD terms beside the per-tet elastic kernel; ACCD beside the
  // line search's first energy).  Forked from and joined back into `stream`
  // with events, so the caller still sees one stream.
  // Set 0 serves the ctx stream; sets 1..3 serve the capture streams
  // cap[0..2] (a stream pulled into one graph capture cannot join another
  // while that capture is open).
  cudaStream_t side[4][2] = {};
  cudaEvent_t ev_fork[4] = {};
  cudaEvent_t ev_join[4][2] = {};
  // CUDA graphs (ipc_set_graph_mode): 1 = each PCG solve is one graph (a
  // WHILE node over one iteration), 2 = the whole step is one graph
  int graph_mode = 0;
  cudaGraphExec_t pcg_exec = nullptr;
  cudaGraphExec_t step_exec = nullptr;
  cudaGraphExec_t roll_exec = nullptr;  // ipc_rollout's graph
  int pcg_iter_launches = 0;      // kernel launches per PCG iteration
  bool pcg_graph_pending = false; // a graph solve ran; its iteration count is not yet read
  struct StepLaunches {           // launches per section of the step graph, counted at capture
    long long pre = 0, newton = 0, pcg_iter = 0, ls_prep = 0, ls_trial = 0, post = 0;
  } step_launches;
  struct RollLaunches {           // the same for the rollout graph
    long long pre = 0, iter = 0, pcg_iter = 0, ls_prep = 0, ls_trial = 0;
  } roll_launches;
  bool roll_pending = false;      // a rollout ran; its results are not yet read
  long long last_loop_iters = 0, last_pcg_launches = 0;  // of the last graph step / rollout
  cudaStream_t cap[3] = {nullptr, nullptr, nullptr};  // capture streams of conditional bodies
  unsigned int* h_step_ctl = nullptr;  // pinned read-back of Dev::step_ctl (8)
  // the last ipc_step: its envs, start time, and whether its results (and,
  // for a graph step, its launch count) are still to be read
  std::vector<int> last_sel;
  std::chrono::steady_clock::time_point step_t0;
  bool step_pending = false, step_graph_pending = false;
  int n_sm = 148;
  // profiling
  bool prof_on = false;
  long long launches = 0;
  std::vector<long long> prof_launches;
  std::vector<double> prof_ms;
  std::vector<cudaEvent_t> ev_free;
  struct Pend { int kind; cudaEvent_t a, b; };
  std::vector<Pend> pending;
};
