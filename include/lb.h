/*
 * lb.h — C ABI of the GB300 fluctuating D3Q19 lattice-Boltzmann + bead-spring chain library
 * (libgblb.so).
 *
 * The method is the explicit-solvent model of Pham, Schiller, Prakash & Duenweg,
 * "Implicit and explicit solvent models for the simulation of a single polymer chain in
 * solution: Lattice Boltzmann vs Brownian dynamics" (arXiv:0903.5067), Sec. II:
 *   - fluid: fluctuating lattice Boltzmann equation (Sec. II B, Eq. 3) on D3Q19 with the
 *     second-order equilibrium (Eq. 4), moment-space relaxation and noise on every
 *     non-conserved mode ("full thermalization"), periodic cubic box of L^3 nodes;
 *   - chain: N beads, FENE bonds and WCA (Lennard-Jones cut at 2^(1/6) sigma, shifted) between
 *     all monomers (Sec. II A, Eqs. 1-2);
 *   - coupling: flow velocity interpolated from the 8 surrounding nodes, Stokes friction
 *     -zeta_bare (v - u) plus a balancing Langevin force, reaction spread back onto the same
 *     nodes so that momentum is conserved (Sec. II B, last paragraph).
 *
 * Units: all physical arguments are in the caller's (MD) unit system; nodes sit at
 * positions a*(x, y, z), x, y, z in [0, L).  Populations are partial mass densities.
 *
 * Conventions for every call:
 *   - returns an lb_status (0 = LB_OK); lb_strerror() names it;
 *   - host buffers are caller-owned; every output buffer comes with its capacity in
 *     elements and the call fails with LB_ERR_ARG when it is too small;
 *   - device work is enqueued on the context's stream (lb_set_stream; default: the legacy
 *     default stream); calls that return data to the host synchronise that stream;
 *   - errors found on the device (broken FENE bond, non-finite state) are latched in a
 *     device status word and returned by the next synchronising call (lb_sync, lb_get_*).
 *   - one context = one fluid box + at most one chain, used from one host thread at a time.
 */
#ifndef GBLB_LB_H
#define GBLB_LB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_ctx lb_ctx; /* opaque, library-owned */

enum lb_status {
  LB_OK = 0,
  LB_ERR_ARG = 1,       /* invalid argument or buffer too small */
  LB_ERR_CUDA = 2,      /* a CUDA runtime call failed */
  LB_ERR_OOM = 3,       /* device allocation failed */
  LB_ERR_FENE = 4,      /* a FENE bond reached r >= R0 (Sec. II A, Eq. 1 diverges) */
  LB_ERR_NONFINITE = 5, /* NaN/Inf in the fluid or bead state */
  LB_ERR_TIMEOUT = 6,   /* a bounded device-side wait gave up */
  LB_ERR_STATE = 7      /* call not valid in the context's current state */
};

/* Storage/arithmetic precision of a context.
 * LB_FP64: populations stored as full n_i in FP64, FP64 arithmetic (the plain path).
 * LB_FP32: populations stored as deviations n_i - w_i rho0 in FP32, FP32 arithmetic.
 * LB_BF16 / LB_FP16: deviations stored in 16 bits, FP32 arithmetic. */
enum lb_precision { LB_FP64 = 0, LB_FP32 = 1, LB_BF16 = 2, LB_FP16 = 3 };

/* Create a fluid box (Sec. II B).  L >= 4 nodes per side; rho (background mass density
 * rho0), eta (shear viscosity), eta_b (bulk viscosity), h (time step, LB and MD) and a
 * (lattice spacing) > 0; kT >= 0.  The relaxation eigenvalues gamma_s, gamma_b derived from
 * eta, eta_b must lie in (-1, 1) (always true for positive viscosities).  seed keys the
 * Philox noise streams (its low 32 bits).  The fluid starts at rest, n_i = w_i rho0.
 * No device memory is touched until the first device call.  *out receives the context. */
int lb_create(lb_ctx** out, int L, double rho, double eta, double eta_b, double kT, double h,
              double a, uint64_t seed, int precision);

/* Add the bead-spring chain (Sec. II A-B): N beads of mass m, friction zeta (zeta_bare),
 * FENE (k_fene, R0), WCA (eps, sigma).  x0: 3N positions (bead-major x,y,z; unwrapped) or
 * NULL to let the library generate a walk of step `bond` starting at the box centre
 * (self-avoiding when saw != 0: no bead closer than sigma to an earlier non-adjacent one);
 * v0: 3N velocities or NULL for zero.  1 <= N <= 1024.  Must precede the first device
 * call.  Bonds initially at r >= R0 give LB_ERR_FENE. */
int lb_add_chain(lb_ctx* ctx, int N, double m, double zeta, double k_fene, double R0, double eps,
                 double sigma, const double* x0, const double* v0, double bond, int saw);

/* Run-time options.  noise_fluid / noise_beads switch the fluctuating terms (both also off
 * when kT = 0); stress_only restricts fluid noise to the six stress modes (the original
 * Ahlrichs-Duenweg thermalization, Table 1 note b); ext_bead_force (3 doubles or NULL) is a
 * constant force on every bead; counter_force_fluid != 0 adds the uniform force density
 * -N ext_bead_force / (L a)^3 to every node so that total momentum stays conserved. */
int lb_set_options(lb_ctx* ctx, int noise_fluid, int noise_beads, int stress_only,
                   const double ext_bead_force[3], int counter_force_fluid);

/* Multiple time stepping (Sec. II E: MD step 0.01, LB step 0.02): n MD steps of length h/n
 * per LB step of length h (lb_create's h), the beads seeing the frozen post-stream fluid and
 * the fluid receiving their reaction averaged over the LB step.  n = 1 (default): LB step =
 * MD step.  1 <= n <= 16 and 8 N n <= 16384; only before the first device call. */
int lb_set_md_substeps(lb_ctx* ctx, int n);

/* Device stream (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream); NULL =
 * legacy default stream.  Must name a stream of the current device. */
int lb_set_stream(lb_ctx* ctx, void* stream);

/* Device workspace: size in bytes (valid after lb_add_chain, if any) and binding of a
 * caller-owned device buffer of at least that size, 256-byte aligned, on the current
 * device, that the caller keeps alive until lb_destroy.  Without a binding the library
 * allocates (cudaMalloc) and frees the workspace itself. */
int lb_workspace_size(lb_ctx* ctx, size_t* bytes);
int lb_bind_workspace(lb_ctx* ctx, void* device_ptr, size_t bytes);

/* Advance n >= 0 coupled steps (Sec. II B, Eq. 3 for the fluid; velocity Verlet for the
 * beads, friction at the half-step velocity).  Asynchronous on the context stream.  The force
 * correction of the last step is kept pending (the next step reads it where it pulls); every
 * call that reads or replaces the fluid state (populations, observables, checkpoints, the
 * adjoint) applies it first, so results never depend on how steps are split into calls. */
int lb_step(lb_ctx* ctx, int64_t n);

/* Wait for the context stream and return the latched device status. */
int lb_sync(lb_ctx* ctx);

/* Full populations n_i (FP64, mass densities), layout [i][z][y][x], 19 L^3 values, in the
 * ABI velocity order (0; +x,-x,+y,-y,+z,-z; (1,1,0),(-1,-1,0),(1,-1,0),(-1,1,0),(1,0,1),
 * (-1,0,-1),(1,0,-1),(-1,0,1),(0,1,1),(0,-1,-1),(0,1,-1),(0,-1,1)), post-collision and
 * force-corrected, as they stand between two steps.  Synchronising. */
int lb_get_populations(lb_ctx* ctx, double* out, size_t cap);
/* Replace the populations (same layout, 19 L^3 doubles).  Enqueued on the stream. */
int lb_set_populations(lb_ctx* ctx, const double* in, size_t count);

/* Bead positions (unwrapped) and velocities, 3N each (bead-major).  Either pointer may be
 * NULL.  Synchronising.  Before the first device call it returns the staged initial chain
 * (given or generated by lb_add_chain) without touching the device. */
int lb_get_beads(lb_ctx* ctx, double* x, double* v, size_t cap);
/* The same read-back without waiting, so that the caller can keep steps queued while earlier
 * results travel: it follows everything enqueued on the context stream before the call, and
 * its copies (from a snapshot the bead kernel writes at the end of every step) run on the
 * library's own stream, so that steps enqueued afterwards proceed meanwhile.  x, v (3N
 * doubles each, v may be NULL) must stay valid until the read-back completes and should be
 * pinned (page-locked) host memory for the copies to be asynchronous.  *ticket identifies the
 * read-back; lb_wait(ctx, ticket) blocks until it (and everything enqueued on the context
 * stream before it) has completed and returns the device status latched at that point.
 * Read-backs complete in the order they were asked for; tickets older than the last 8 remain
 * valid.  Needs a chain and a live context (LB_ERR_ARG otherwise: a bad pointer, size or
 * ticket). */
int lb_get_beads_async(lb_ctx* ctx, double* x, double* v, size_t cap, int64_t* ticket);
int lb_wait(lb_ctx* ctx, int64_t ticket);

/* FP64 observables (Sec. III A-B), cap >= LB_NOBS:
 *  [0] step  [1] mass a^3 sum n  [2..4] total momentum (fluid + beads + h/2 sum F_c)
 *  [5..7] fluid momentum  [8] R_g^2  [9] R_e^2  [10..12] centre of mass (unwrapped)
 *  [13] g1: mean |r_i(t) - r_i(t0)|^2 of the two innermost beads  [14] g3: |R_cm(t) -
 *  R_cm(t0)|^2  [15] bead kinetic temperature m<v^2>/3  [16] count of non-positive node
 *  densities met by the noise  [17] number of accumulated samples  [18] <R_g^2> and
 *  [19] <R_e^2> over the samples.  t0 is the chain's state when it was added (or at the
 *  last lb_reset_reference).  Synchronising. */
#define LB_NOBS 20
int lb_get_observables(lb_ctx* ctx, double* out, size_t cap);
/* Accumulate <R_g^2>, <R_e^2> every `stride` steps inside lb_step (0 = off). */
int lb_set_obs_stride(lb_ctx* ctx, int stride);
/* Take the current bead positions as the reference t0 of g1 and g3; clear accumulators. */
int lb_reset_reference(lb_ctx* ctx);

/* Trajectory recording for the observables of Sec. III A/B (g1, g2, g3, Rouse modes,
 * S(k), S(k,t); see the lb_analysis_* functions below).  traj_dev: caller-owned device
 * memory for `capacity` frames of 3N doubles (unwrapped positions, [frame][bead][xyz]),
 * used as a ring: frame f is stored at slot f mod capacity.  Frame 0 is the current state,
 * written at this call; then one frame after every `stride` steps of lb_step.  A NULL
 * buffer, capacity <= 0 or stride <= 0 stops recording.  LB_ERR_STATE without a chain.
 * The library writes the buffer on its stream; read it after lb_sync. */
int lb_record_trajectory(lb_ctx* ctx, double* traj_dev, int capacity, int stride);
/* Frames recorded since the last lb_record_trajectory (the ring keeps the last capacity). */
int lb_trajectory_frames(lb_ctx* ctx, int64_t* frames);

/* Gradient of a chain observable through T coupled steps, by the adjoint of the step with
 * the noise held fixed (same Philox streams forward and backward).  Observable:
 * O = sum_b |x_b(T) - x_b(0)|^2 (unwrapped positions).  Gradients with respect to the
 * initial bead positions x_b(0) (grad_x0, 3N, bead-major) and to zeta_bare (grad_zeta).
 * The forward run keeps full-state checkpoints every K steps and recomputes each segment
 * during the reverse sweep (memory ~ (T/K + K) states).  Must be called on a context that
 * has not stepped yet (the initial force is F_cons(x_0)); requires a chain, one MD step per
 * LB step and no fluid body force (LB_ERR_STATE otherwise); leaves the context at step T.  Allocates its checkpoint and adjoint memory with
 * cudaMalloc for the duration of the call. */
int lb_adjoint_displacement(lb_ctx* ctx, int64_t T, int K, double* objective, double* grad_x0,
                            size_t cap, double* grad_zeta);

/* Checkpoint / resume: parameters, options, step counter, populations (storage precision),
 * bead state.  Noise is counter-based, so a resumed run continues bit-identically. */
int lb_save(lb_ctx* ctx, const char* path);
int lb_load(lb_ctx* ctx, const char* path);

/* Step counter and device kernel timing: when enabled, lb_step records CUDA events around
 * every fused LB launch; lb_get_timing returns their summed duration (ms) and count. */
int64_t lb_get_step(lb_ctx* ctx);
int lb_set_timing(lb_ctx* ctx, int enable);
int lb_get_timing(lb_ctx* ctx, double* total_ms, int64_t* launches);

/* Wait for the context's outstanding work and read-backs, then free its device memory
 * (a caller-bound workspace stays the caller's) and the handle.  NULL is ignored. */
void lb_destroy(lb_ctx* ctx);
/* A static, NUL-terminated name for a status code ("unknown status" for others). */
const char* lb_strerror(int status);
/* The message of the calling thread's last failing single-context call (lb_create ..
 * lb_adjoint_displacement, the status a synchronising call reports included), copied
 * NUL-terminated into buf (truncated to cap - 1 bytes; buf may be NULL) and then cleared;
 * returns its full length, 0 when there is none.  Batch and Brownian-dynamics calls return
 * their status without a message. */
size_t lb_last_error(char* buf, size_t cap);

/* --- test hooks on raw device buffers (enqueued on `stream`, no context) --------------- */

/* Philox4x32-10 on n counters: ctr_dev[4n] -> out_dev[4n] (uint32), key (k0, k1). */
int lb_philox4x32_10(const uint32_t* ctr_dev, int64_t n, uint32_t k0, uint32_t k1,
                     uint32_t* out_dev, void* stream);

/* Cell index of FP32 coordinates: out_dev[i] = floor(x_dev[i] / a) mod L in [0, L), the
 * quotient rounded once in FP32 (the bead kernel's own index function). */
int lb_cell_index_f32(const float* x_dev, int64_t n, float a, int L, int32_t* out_dev,
                      void* stream);

/* Test hook: the coupling's cells as the bead kernel of the last step used them (Sec. II B,
 * last paragraph: the 8 nodes around each bead).  nodes receives the 8 N s corner nodes of
 * the last step's s MD substeps, entry 8 (s' N + b) + c for substep s', bead b and corner
 * c = dx + 2 dy + 4 dz (node index x + L (y + L z)); x_stored receives the 3 N stored
 * coordinates (high part of the compensated position, wrapped into [0, L a), in the
 * context's arithmetic precision, as doubles) from which the last substep took its cells.
 * cap >= 8 N s for nodes and >= 3 N for x_stored (either pointer may be NULL).  Needs a chain
 * (LB_ERR_STATE) and a stepped context; synchronising. */
int lb_debug_coupling_cells(lb_ctx* ctx, int32_t* nodes, double* x_stored, size_t cap);

/* --- batched replicas ------------------------------------------------------------------
 * R independent boxes advanced in lockstep by one launch per kernel stage (the ensemble of
 * box sizes and chain lengths the paper runs for its finite-size and cost studies, Sec. II E,
 * Sec. III B-C).  Replica r has L[r] nodes per side (4..256), a chain of N[r] beads (0..1024)
 * whose 3N[r] positions are concatenated in x0 (replica order; NULL only if every N[r] = 0),
 * and its own noise stream: Philox key (seeds[r] low 32 bits, tag | r << 8).  Fluid and chain
 * parameters as in lb_create / lb_add_chain, shared by all replicas; md_substeps as in
 * lb_set_md_substeps.  precision: LB_FP32 or LB_FP64.  Workspace, stream and errors as for a
 * context. */
typedef struct lb_batch lb_batch;
int lb_batch_create(lb_batch** out, int R, const int* L, const int* N, const uint64_t* seeds,
                    double rho, double eta, double eta_b, double kT, double h, double a, double m,
                    double zeta, double k_fene, double R0, double eps, double sigma,
                    const double* x0, int precision, int md_substeps);
int lb_batch_set_stream(lb_batch* b, void* stream);
int lb_batch_workspace_size(lb_batch* b, size_t* bytes);
int lb_batch_bind_workspace(lb_batch* b, void* device_ptr, size_t bytes);
/* Noise switches of every replica, as lb_set_options (stress_only: noise on the six stress
 * modes only, the thermalization of Table 1 note b).  Only before the batch's workspace is
 * bound by its first use (step, autotune, read); LB_ERR_STATE after. */
int lb_batch_set_options(lb_batch* b, int noise_fluid, int noise_beads, int stress_only);
/* Tile size of the batched LB kernel (128, 256 or 512 threads) and persistent thread blocks
 * per SM (0 = one block per tile).  Results do not depend on the shape. */
int lb_batch_set_shape(lb_batch* b, int threads, int blocks_per_sm);
/* Measure every shape for a few steps, keep the fastest and return it; the trial steps are
 * undone (the replicas restart from their initial state).  Only before the first step. */
int lb_batch_autotune(lb_batch* b, int* threads, int* blocks_per_sm);
/* Advance every replica n steps; runs of 16 steps are replayed from a captured CUDA graph. */
int lb_batch_step(lb_batch* b, int64_t n);
int lb_batch_sync(lb_batch* b);
int lb_batch_get_populations(lb_batch* b, int r, double* out, size_t cap);
int lb_batch_get_beads(lb_batch* b, int r, double* x, double* v, size_t cap);
int lb_batch_get_observables(lb_batch* b, int r, double* out, size_t cap);
int64_t lb_batch_nodes(lb_batch* b); /* total nodes of all replicas */
/* Add the current R_g^2, R_e^2 of every replica to its FP64 accumulators; read the means
 * with lb_batch_get_observables (entries 17..19). */
int lb_batch_accumulate(lb_batch* b);
void lb_batch_destroy(lb_batch* b);

/* --- chain observables on a device trajectory (Sec. III A and III B) ----------------------
 * traj: T frames of N beads, [t][n][xyz] FP64 unwrapped positions on the current device
 * (e.g. the ring of lb_record_trajectory, unrolled to oldest-first).  Outputs are
 * caller-owned device arrays, written on `stream` (a cudaStream_t, NULL = legacy default);
 * nothing is allocated and nothing synchronises.  Averages over time origins use every
 * origin t0 with t0 + lag < T.  Every output element is a fixed-order sum, so results are
 * reproducible bit for bit.  Invalid sizes or pointers return LB_ERR_ARG.
 *
 * lb_analysis_msd: out[3][max_lag+1] = g1, g2, g3 at lags 0..max_lag: the mean-square
 *   displacement of monomers i0 and i1 (averaged over both; the paper uses the two innermost
 *   monomers), the same in the centre-of-mass frame, and of the centre of mass (Sec. III B).
 * lb_analysis_rouse_modes: X[T][P][3], X_p(t) = (1/N) sum_{n=1..N} r_n(t) cos(p pi (n-1/2)/N)
 *   for p = 1..P, P <= N-1 (Sec. III B, Rouse modes).
 * lb_analysis_rouse_correlation: c[P][max_lag+1] = < X_p(t0+lag) . X_p(t0) >; c[p][0] is
 *   <X_p^2>, the normalisation of the paper's correlation function.  max_lag <= 65535.
 * lb_analysis_static_sk: S[nk] = (1/N) sum_{i,j} < sin(k r_ij) / (k r_ij) > over the T
 *   frames, for the nk wave numbers k[] (device array) (Sec. III A, S(k)).
 * lb_analysis_inverse_radius: out[0] = <1/R_H> = (1/N^2) sum_{i != j} <1/r_ij> over the T
 *   frames (Sec. III A, the hydrodynamic radius of the chain in an infinite medium); N >= 2
 *   and no two beads at the same position.
 * lb_analysis_dynamic_sk: S[nk][max_lag+1] = (1/N) sum_{i,j} < sin(k d)/(k d) >,
 *   d = |r_i(t0+lag) - r_j(t0)|, over origins t0 = 0, s, 2s, ... (s = origin_stride)
 *   (Sec. III B, S(k,t); the isotropic average of exp(i k.[r_i(t) - r_j(0)])). */
int lb_analysis_msd(const double* traj, int T, int N, int max_lag, int i0, int i1, double* out, void* stream);
int lb_analysis_rouse_modes(const double* traj, int T, int N, int P, double* X, void* stream);
int lb_analysis_rouse_correlation(const double* X, int T, int P, int max_lag, double* c, void* stream);
int lb_analysis_static_sk(const double* traj, int T, int N, const double* k, int nk, double* S, void* stream);
int lb_analysis_inverse_radius(const double* traj, int T, int N, double* out, void* stream);
int lb_analysis_dynamic_sk(const double* traj, int T, int N, const double* k, int nk, int max_lag,
                           int origin_stride, double* S, void* stream);

/* --- Brownian dynamics with hydrodynamic interaction (Sec. II C) -----------------------------
 * `replicas` independent chains of N beads in an infinite medium, advanced by the Ito-Euler
 * update r += (D/kT) F dt + sqrt(2 dt) B.W with D/kT = zeta^-1 1 on the diagonal blocks and the
 * regularised Rotne-Prager-Yamakawa tensor (Stokes radius zeta / (6 pi eta_s)) between beads
 * (hi = 0: free draining), B.W from Fixman's Chebyshev expansion of sqrt(D) of the given
 * degree (1..64) on spectral bounds from `power_iters` power iterations per step.  Forces:
 * FENE bonds (k_fene, R0) and WCA (eps, sigma) between all pairs.  Units as given (the
 * paper's comparison uses MD/LB units with zeta = zeta_eff, Sec. II D).  Noise: Philox4x32-10,
 * key (seed, 3 | replica << 8), counter (step, bead, 0, 0).  x0: replicas x N x 3 doubles.
 * precision: LB_FP64 (N <= 52) or LB_FP32 (N <= 74) arithmetic; positions are kept in FP64.
 * The library allocates its device memory; work runs on the stream set with lb_bd_set_stream.
 * lb_bd_get_beads copies all replicas' positions (replicas x N x 3) and synchronises; a FENE
 * bond at or beyond R0 is reported as LB_ERR_FENE by lb_bd_sync and lb_bd_get_beads. */
typedef struct lb_bd lb_bd;
int lb_bd_create(lb_bd** out, int replicas, int N, double kT, double zeta, double eta_s, double dt,
                 double k_fene, double R0, double eps, double sigma, int hi, int degree, int power_iters,
                 uint64_t seed, const double* x0, int precision);
int lb_bd_set_stream(lb_bd* b, void* stream);
int lb_bd_step(lb_bd* b, int64_t n);
int lb_bd_sync(lb_bd* b);
int lb_bd_get_beads(lb_bd* b, double* x, size_t cap);
int64_t lb_bd_get_step(lb_bd* b);
void lb_bd_destroy(lb_bd* b);

/* --- allocation-free variant ---------------------------------------------------------
 * Fluid mass and momentum of a population field, like lb_get_observables' entries [1] and
 * [5..7], for callers that cannot allocate device memory where they need these sums: a host
 * application whose device memory is all reserved by another allocator (a framework's
 * caching allocator or a pool sized to the whole GPU), where an allocation of the library's
 * own would fail or fragment that pool; and time-critical loops, where cudaFree's implicit
 * device-wide synchronisation and an allocation's latency are not acceptable.  The paper has
 * no counterpart; this is a service of the library.
 *
 * pop_dev: 19 L^3 full populations (FP64, mass densities) on the current device, in the
 * layout lb_get_populations returns ([i][z][y][x], ABI velocity order).  out_host receives
 * 4 doubles: a^3 sum n, then (a^4/h) sum_i n_i c_i (x, y, z).  stream: a stream of the
 * current device (NULL: the default stream); the two kernels and the copy of the result
 * to out_host are enqueued on it, and the call synchronises that stream before it returns.
 *
 * Scratch: a file-scope device array of LB_NOALLOC_MAX_L^3 / 256 partial sums (2 MiB), held by
 * every GPU that loads the library until the process exits; L > LB_NOALLOC_MAX_L returns
 * LB_ERR_ARG.  The function calls no cudaMalloc, cudaFree or allocating library routine.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current and keeps it for later calls; make that first call before any
 * stream capture begins.  The kept address does not survive cudaDeviceReset of that device
 * (do not call this function again in a process that reset the device).  All calls share the
 * array (it keeps the last call's partial sums; each call overwrites every slot it reads),
 * so calls that overlap on the GPU, from several streams or threads, race.
 * Errors: LB_ERR_ARG for null pointers, a, h <= 0, L outside [1, LB_NOALLOC_MAX_L] or a
 * stream of another device; LB_ERR_CUDA when a launch, the copy or the synchronisation
 * fails.  Every failure leaves its reason for lb_last_error. */
#define LB_NOALLOC_MAX_L 256
int lb_fluid_sums_noalloc(const double* pop_dev, int L, double a, double h, double* out_host,
                          void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GBLB_LB_H */
