// Launch wrappers of the ABD-IPC kernels (host-callable).
#pragma once

#include "ctx.h"

namespace ipc {

// env masks passed to kernels: the EnvInt flag that must be non-zero
// (I_SEL, I_ACTIVE, I_PCG, I_LS) for an env to be processed.

// ---- contact (kernels_contact.cu)
int launch_cv_pos(const Dev& d, int flag, bool with_disp, cudaStream_t s);
int launch_obj_box(const Dev& d, int flag, bool swept, cudaStream_t s);
int launch_broad(const Dev& d, int flag, bool swept, cudaStream_t s);
int launch_barrier(const Dev& d, int flag, cudaStream_t s);
int launch_accd(const Dev& d, cudaStream_t s);
// lagged friction (no launches when friction_mu = 0)
int launch_fric_setup(const Dev& d, cudaStream_t s);
int launch_fric_assemble(const Dev& d, cudaStream_t s);
int launch_fric_spmv(const Dev& d, cudaStream_t s);
int launch_fric_energy(const Dev& d, int use_alpha, cudaStream_t s);
int launch_pair_energy(const Dev& d, int use_alpha, cudaStream_t s);
int launch_min_dist(const Dev& d, int flag, cudaStream_t s);
// crossing surfaces of I_SEL-style flagged envs -> I_FLAG = 2 (needs cvx and primitive boxes)
int launch_cross_check(const Dev& d, int flag, cudaStream_t s);
int launch_pnorm_body(const Dev& d, cudaStream_t s);

// ---- solver (kernels_solver.cu)
int launch_predict(const Dev& d, int flag, cudaStream_t s);
int launch_attach_targets(const Dev& d, int flag, cudaStream_t s);
int launch_tet(const Dev& d, cudaStream_t s);
int launch_body(const Dev& d, cudaStream_t s);
int launch_assemble(const Dev& d, cudaStream_t s);
int launch_grad(const Dev& d, cudaStream_t s);
int launch_precond(const Dev& d, cudaStream_t s);
// ---- PCG (kernels_pcg.cu)
int launch_pcg_init(const Dev& d, cudaStream_t s);
// work list of the envs whose I_PCG flag is set; with use_cond the kernel
// sets the graph condition `h` (1 while an env iterates)
int launch_pcg_begin(const Dev& d, cudaStream_t s, cudaGraphConditionalHandle h, int use_cond);
// one PCG iteration = mat-vec (+ friction mat-vec) + update; the update's
// last CTA advances the iteration counter and, with use_cond, sets `h`
int launch_pcg_matvec(const Dev& d, cudaStream_t s);
int launch_pcg_pairs(const Dev& d, cudaStream_t s);
int launch_pcg_iter(const Dev& d, cudaStream_t s, cudaGraphConditionalHandle h, int use_cond, unsigned window);
int launch_debug_set_updk(const Dev& d, int env, int v, cudaStream_t s);
int pcg_iter_ctas_per_sm(int prec, int unroll, int bound, bool fr);
int pcg_multi_ctas_per_sm(int prec, int unroll, bool fr);
int pcg_iters_per_launch(const Dev& d, unsigned window);
int launch_pcg_update(const Dev& d, cudaStream_t s, cudaGraphConditionalHandle h, int use_cond,
                      unsigned window = 0xffffffffu);
// resident 128-thread CTAs per SM of the PCG kernels (grid = 148 x this)
int pcg_ctas_per_sm(int prec, int unroll);
// diagnostics: PCG direction from the FP64 rows in Dev::z; q back to Dev::q
int launch_debug_dir_from_rows(const Dev& d, cudaStream_t s);
int launch_debug_q_to_rows(const Dev& d, cudaStream_t s);
int launch_newton_check(const Dev& d, cudaStream_t s);   // pnorm / cres (rows)
int launch_newton_decide(const Dev& d, cudaStream_t s);
int launch_al_update(const Dev& d, cudaStream_t s);
int launch_ls_init(const Dev& d, cudaStream_t s);
int launch_energy(const Dev& d, int use_alpha, int which /*0: E0, 1: E1*/, cudaStream_t s);
int launch_ls_decide(const Dev& d, cudaStream_t s);
int launch_ls_apply(const Dev& d, cudaStream_t s);
int launch_finalize(const Dev& d, cudaStream_t s);
// rollout (each env runs its own sequence of steps inside one device loop)
int launch_roll_setup(const Dev& d, const double* table, int n_steps, unsigned long long cap, cudaStream_t s);
int launch_roll_init(const Dev& d, cudaStream_t s);
int launch_roll_begin(const Dev& d, cudaStream_t s);
int launch_roll_end(const Dev& d, cudaStream_t s);
int launch_roll_cond(const Dev& d, cudaStream_t s, cudaGraphConditionalHandle h);
int launch_env_reset(const Dev& d, int what, cudaStream_t s);
int launch_check_overflow(const Dev& d, cudaStream_t s);
// loop control of the device-side step (k_flag_cond in kernels_solver.cu)
int launch_flag_cond(const Dev& d, cudaStream_t s, int flag, int cnt, int inc, int acc, int rst, unsigned cap,
                     cudaGraphConditionalHandle h, int use_cond);
int launch_check_inverted(const Dev& d, cudaStream_t s);
int launch_scatter_targets(const Dev& d, cudaStream_t s);
int launch_gather_coated(const Dev& d, cudaStream_t s);

// element kernels on caller buffers
int launch_k_tet(int n, const double* x, const double* Dmi, const double* vol, double mu, double lam,
                 double* E, double* g, double* H, int project, cudaStream_t s);
int launch_k_barrier(int n, const double* X, const int* is_ee, const double* w, const double* eps,
                     double dhat, double* E, double* g, double* H, int project, cudaStream_t s);
int launch_k_accd(int n, const double* X0, const double* P, const int* is_ee, double sfrac, int max_iter,
                  double* toi, int* iters, cudaStream_t s);

}  // namespace ipc
