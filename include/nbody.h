/*
 * nbody.h -- C ABI of the GB300 (sm_103a) all-pairs N-body library.
 *
 * The library evaluates the O(N^2) direct-summation forces of Elsen et al.,
 * "N-Body Simulations on GPUs" (arXiv 0706.3060) -- softened gravity (Eq. 1,
 * Table 1 "Gravity (accel)") and Lennard-Jones plus Coulomb in a continuum
 * solvent of constant dielectric (Table 1 "LJC(constant)") -- and the update
 * step that consumes them (Sec. 1 splits each time step into a force
 * evaluation and an update), which it implements as kick-drift-kick leapfrog.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Interactions are ordered pairs (i, j), i != j, as in Sec. 2: the force on
 *    i sums over all j. One-sided tiles evaluate each ordered pair for its
 *    target, as the paper does; Newton-symmetric tiles (NBODY_TILE_SYMMETRIC,
 *    the tuned choice at mid and large N for gravity, LJC, their VJPs,
 *    acceleration + jerk and batched ensembles) evaluate each unordered pair
 *    once and apply it to both particles, the pair terms being antisymmetric
 *    (or, for the sigma/epsilon derivatives, symmetric) under the swap. Both
 *    give the same sums up to FP32 rounding order and are each reproducible.
 *  - Particle data are arrays of float4, 16-byte aligned, one element per
 *    particle:
 *      pos_m[i] = (x, y, z, m)                          both laws
 *      prm[i]   = (q~, s~, e~, type)                    LJC only, made by
 *                 nbody_pack_ljc: q~ = q sqrt(k_e/eps_r), s~ = sigma/2,
 *                 e~ = sqrt(24 eps); type is the atom type as a float.
 *      acc[i]   = (ax, ay, az, phi)  acceleration and per-particle potential
 *                 (gravity: phi_i = -G sum_j m_j / s_ij, U = 1/2 sum m_i phi_i;
 *                  LJC: phi_i = sum_j u_ij pair energies, U = 1/2 sum phi_i).
 *      vel[i]   = (vx, vy, vz, unused)
 *  - Pointers are device pointers unless an entry point says otherwise. The
 *    caller owns every array it passes; the library owns only its internal
 *    workspace (see nbody_release).
 *  - All work is enqueued on the caller's CUDA stream `stream` (a
 *    cudaStream_t; NULL is the legacy default stream) and is asynchronous,
 *    except where a function states that it synchronizes.
 *  - Every function returns an nbody_status. On failure the reason is
 *    available from nbody_last_error() (thread-local). No function aborts,
 *    exits or throws across the ABI. Arguments are validated before any work
 *    is enqueued; a rejected call leaves every output untouched.
 *  - A kernel never waits without a bound: a wait that runs out sets a device
 *    error flag, the kernel returns, and the next synchronizing call reports
 *    NBODY_ETIMEOUT.
 */
#ifndef NBODY_H
#define NBODY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *nbody_stream_t; /* identical to cudaStream_t */

typedef enum {
    NBODY_OK = 0,
    NBODY_EINVAL = 1,       /* bad size, null pointer, bad enum or flag      */
    NBODY_EALIGN = 2,       /* pointer not 16-byte aligned                   */
    NBODY_ENOMEM = 3,       /* workspace allocation failed                   */
    NBODY_ECUDA = 4,        /* a CUDA runtime call failed                    */
    NBODY_ETIMEOUT = 5,     /* a bounded device wait ran out                 */
    NBODY_EUNSUPPORTED = 6, /* no GPU, wrong architecture, or unsupported mode */
} nbody_status;

/* Force laws (Table 1). */
enum {
    NBODY_LAW_GRAV = 0,       /* "Gravity (accel)", Eq. 1                          */
    NBODY_LAW_LJC = 1,        /* "LJC(constant)": LJ 12-6 + Coulomb / eps_r         */
    NBODY_LAW_LJC_LINEAR = 2, /* "LJC(linear)": LJ 12-6 + Coulomb with a dielectric
                                 growing linearly with distance, energy
                                 kq q_i q_j / r^2 (kq = k_e / D, packed into prm
                                 by nbody_pack_ljc), force 2 kq q_i q_j r_ij / r^4.
                                 Every entry point that takes a law accepts it
                                 except the jerk and Hermite calls.             */
};

/* nbody_params.flags */
enum {
    NBODY_COMPUTE_POT = 1u << 0,     /* also compute phi (acc[i].w)            */
    NBODY_PRECISE_RSQRT = 1u << 1,   /* one Newton step on the hardware rsqrt  */
    NBODY_NO_COMPENSATION = 1u << 2, /* plain FP32 sums (default: per-tile
                                        TwoSum compensated sums, and the
                                        per-slice or per-block partials added
                                        with compensation); Newton-symmetric
                                        tiles always sum within a block pair
                                        plainly, and with this flag also add
                                        their per-block partials plainly      */
    NBODY_ACC_VALID = 1u << 3,       /* nbody_step: acc already holds a(x) for
                                        the entry positions                    */
    NBODY_ACCUMULATE = 1u << 4,      /* nbody_adjoint: add into the outputs    */
    NBODY_FIXED_POINT = 1u << 5,     /* gravity, eps > 0, nbody_forces/step:
                                        64-bit fixed-point accumulation of the
                                        per-tile sums (Sec. 3.2, GRAPE-6);
                                        results are bitwise independent of the
                                        j-split. params->tile then indexes
                                        tile table 4. nbody_adjoint(_leapfrog),
                                        nbody_forces_jerk, nbody_hermite_step:
                                        the Newton-symmetric gravity VJP and
                                        acceleration + jerk tiles add their
                                        per-block partials exactly in fixed
                                        point (64 / 128 B of scratch per
                                        particle); without the flag they do so
                                        only where one partial per block would
                                        pass the partial-sum cap. Other laws or
                                        eps2 == 0: NBODY_EINVAL.               */
};

typedef struct {
    int32_t law;     /* NBODY_LAW_*                                          */
    uint32_t flags;  /* NBODY_* flags above                                  */
    float G;         /* gravitational constant (gravity)                     */
    float eps2;      /* squared softening eps^2 (gravity; the Appendix "eps") */
    int32_t tile;    /* kernel tile configuration, -1 = tuned/default: a row
                        of the law's force table (0-2, 4 with FIXED_POINT);
                        for nbody_adjoint / nbody_adjoint_leapfrog a row of
                        table 5 (gravity VJP), 6 (LJC VJP) or 8 (LJC linear
                        VJP); for
                        nbody_forces_jerk / nbody_hermite_step of table 7  */
    int32_t jsplit;  /* j-slices per i-tile ("replication", Sec. 3.4), 0 = auto */
} nbody_params;

/* Library version (major * 10000 + minor * 100 + patch). Never fails. */
int nbody_version(void);

/* Thread-local message for the last non-OK status returned on this thread. */
const char *nbody_last_error(void);

/* Release the library's internal workspaces on the current device.
 * Synchronizes the device. */
int nbody_release(void);

/* Synchronize `stream`, then report (and clear) any error a kernel recorded
 * since the last check on the current device, by any entry point (including
 * nbody_forces_static): NBODY_ETIMEOUT for a bounded wait that ran out,
 * NBODY_EINVAL for a work item that failed its bounds check. The device error
 * word is a __device__ variable of the library, so recording and reading it
 * allocates nothing. */
int nbody_check(nbody_stream_t stream);

/* Kernel timers. While enabled, every all-pairs kernel launch made outside
 * stream capture is bracketed by two CUDA events recorded on its own stream.
 * nbody_timing_read synchronizes those events and returns, for `which`
 * (0 = force kernels, 1 = VJP kernels), the number of timed launches and their
 * summed device time in milliseconds since the previous read, then resets. */
int nbody_timing_enable(int32_t on);
int nbody_timing_read(int32_t which, int64_t *launches, double *total_ms);

/* Throughput microbenchmark of the units that bound the all-pairs kernels
 * (no counterpart in the paper; used to check the roofline denominators):
 * kind 0 = scalar FP32 FFMA, 1 = packed f32x2 FFMA (2 lane ops each),
 * 2 = MUFU rsqrt, 3 = half FFMA2 / half FFMA chains, 4 = the packed gravity
 * pair loop over shared memory, 5 = the scalar pair loop (kinds 4 and 5 count
 * 12 lane ops per pair). Runs 8 x 256 threads per SM, `iters` iterations;
 * returns lane operations per SM per clock and per second. Synchronizes the
 * device. */
int nbody_peak_probe(int32_t kind, int32_t iters, double *ops_per_clk_sm, double *ops_per_s);

/* Failure-path self test (no counterpart in the paper): enqueues one kernel that
 * waits, with the bounded wait every pipeline uses but limited to limit_cycles
 * (1 .. 1e8), on an mbarrier that nothing completes. The wait runs out, the
 * kernel records NBODY_ETIMEOUT in the error word and returns, and the next
 * nbody_check on `stream` reports NBODY_ETIMEOUT and clears it. Nothing faults
 * or hangs; the context stays usable. */
int nbody_selftest_timeout(int64_t limit_cycles, nbody_stream_t stream);

/* ---------------------------------------------------------------------------
 * Packing (Sec. 2 keeps the coordinates as GPU streams; the Appendix listing
 * reads positions and masses as float4).
 * Converts caller SoA data in double precision into the float4 streams above.
 *   x, y, z, m : n doubles each (device).      pos_m : n float4 (device, out)
 *   nbody_pack_ljc additionally takes q, sigma, eps (per particle, doubles),
 *   type (int32) and kq = k_e / eps_r, and writes prm (n float4).
 * --------------------------------------------------------------------------- */
int nbody_pack_grav(const double *x, const double *y, const double *z, const double *m,
                    void *pos_m, int64_t n, nbody_stream_t stream);
int nbody_pack_ljc(const double *q, const double *sigma, const double *eps,
                   const int32_t *type, double kq, void *prm, int64_t n,
                   nbody_stream_t stream);

/* ---------------------------------------------------------------------------
 * nbody_forces -- one force evaluation (Sec. 2 "forces = kforce(coordinates)",
 * Eq. 1 / Table 1).
 *   pos_m  : n float4 (x, y, z, m)                                   in
 *   prm    : n float4 LJC parameters (NULL for gravity)              in
 *   acc    : n float4 (ax, ay, az, phi); phi only with COMPUTE_POT   out
 *   acc_lo : n float4 low parts of the compensated sums, or NULL     out
 *            (acc + acc_lo is the sum to about twice FP32 precision)
 * Gravity: a_i = G sum_{j!=i} m_j (x_j - x_i) / (|x_j - x_i|^2 + eps2)^{3/2}.
 * LJC    : a_i = F_i / m_i with the 12-6 LJ + Coulomb force of Table 1.
 * Pointers may be device pointers or, all of them together, host pointers; in
 * the host case the library stages through device memory and the call
 * synchronizes `stream` before returning. n == 0 is a no-op. n <= 2^31 - 1.
 * --------------------------------------------------------------------------- */
int nbody_forces(const void *pos_m, const void *prm, void *acc, void *acc_lo, int64_t n,
                 const nbody_params *params, nbody_stream_t stream);

/* nbody_forces_jerk -- acceleration and its time derivative (jerk), Table 1
 * "Gravity (accel & jerk)", the force evaluation of 4th-order Hermite schemes:
 *   a_i = G sum_{j!=i} m_j r / s^3,
 *   j_i = G sum_{j!=i} m_j [ u / s^3 - 3 (r . u) r / s^5 ],
 *   r = x_j - x_i, u = v_j - v_i, s^2 = |r|^2 + eps2.
 *   pos_m, vel : n float4 in; acc, jerk : n float4 out (w = 0). Gravity law only;
 *   NBODY_NO_COMPENSATION is the only accepted flag. Device pointers only. */
int nbody_forces_jerk(const void *pos_m, const void *vel, void *acc, void *jerk, int64_t n,
                      const nbody_params *params, nbody_stream_t stream);

/* nbody_hermite_step -- nsteps fourth-order Hermite predictor-evaluate-correct
 * steps on the acceleration and jerk of nbody_forces_jerk (the integrator Table 1's
 * GAJ kernel serves; Makino & Aarseth 1992):
 *   predict  x_p = x + v dt + a dt^2/2 + j dt^3/6,  v_p = v + a dt + j dt^2/2
 *   evaluate (a1, j1) at (x_p, v_p)
 *   correct  v = v + (a + a1) dt/2 + (j - j1) dt^2/12,
 *            x = x + (v_old + v) dt/2 + (a - a1) dt^2/12
 *   pos_m, vel, acc, jerk : n float4, in/out; acc/jerk hold (a, j) of the exit
 *   state and are read on entry only with NBODY_ACC_VALID. Gravity only.
 *   Device pointers only. */
int nbody_hermite_step(void *pos_m, void *vel, void *acc, void *jerk, int64_t n, float dt,
                       int32_t nsteps, const nbody_params *params, nbody_stream_t stream);

/* nbody_forces_subset -- forces on n_active target particles idx[0..n_active)
 * against all n sources (block time steps, Sec. 3.4: forces on only a subset of
 * the particles at a time). Same laws, flags and accuracy as nbody_forces.
 *   idx : n_active int32 indices into [0, n), device; duplicates allowed
 *   acc : n_active float4 (device): acc[k] = (a, phi) of particle idx[k]
 * The self pair of each target is excluded by its index. An index outside
 * [0, n) is caught on the device (its row is computed for particle 0) and
 * reported by the next nbody_check as NBODY_EINVAL. Device pointers only. */
int nbody_forces_subset(const void *pos_m, const void *prm, const int32_t *idx,
                        int64_t n_active, void *acc, int64_t n, const nbody_params *params,
                        nbody_stream_t stream);

/* nbody_forces_static -- nbody_forces for callers that cannot allocate device
 * memory (a fixed memory budget set at start-up, an allocator owned by another
 * framework, a real-time loop that must not block in cudaMalloc). The paper has
 * no counterpart; it is the same force evaluation, with its scratch in one
 * static __device__ array of 32 MiB inside the library (held by every GPU that
 * loads the library until the process exits) instead of an on-demand
 * workspace. It calls no cudaMalloc, cudaFree or allocating routine.
 *   pos_m, prm, acc, n, params, stream : as in nbody_forces (device pointers
 *   only; no acc_lo; NBODY_COMPUTE_POT, NBODY_PRECISE_RSQRT and
 *   NBODY_NO_COMPENSATION are honoured).
 * Only one-sided tiles run here: an explicit Newton-symmetric tile
 * (NBODY_TILE_SYMMETRIC) is refused with NBODY_EINVAL, and with tile = -1 a
 * tuned symmetric entry is replaced by the law's default one-sided tile. n
 * beyond what the scratch holds (about 699,000 particles for gravity) is
 * rejected with NBODY_EINVAL before any GPU work; at large n the call runs with
 * fewer j-slices than nbody_forces would use, so that the partial sums fit. The
 * first call on each device, with that device current, looks up the array's
 * device address (cudaGetSymbolAddress); make that first call before any stream
 * capture. All calls share the array, which keeps the last call's contents;
 * each call rewrites what it reads, but calls whose GPU work overlaps (e.g. on
 * two streams) race on the array: serialize them. A bounded wait that runs out
 * in its kernels is recorded in the library's device error word (no allocation
 * either) and reported by the next nbody_check, like any other call's. Its
 * kernels are not bracketed by the kernel timers (which create CUDA events). */
int nbody_forces_static(const void *pos_m, const void *prm, void *acc, int64_t n,
                        const nbody_params *params, nbody_stream_t stream);

/* ---------------------------------------------------------------------------
 * nbody_step -- nsteps kick-drift-kick leapfrog steps of size dt (the update
 * step of Sec. 1), each consuming one all-pairs force evaluation:
 *   v += dt/2 a(x);  x += dt v;  v += dt/2 a(x)
 *   pos_m : n float4, in/out; w (mass) is not modified
 *   vel   : n float4, in/out (synchronized with pos_m on entry and exit)
 *   acc   : n float4, in/out: on exit a(x) at the exit positions. On entry it
 *           is read only when params->flags has NBODY_ACC_VALID.
 *   prm   : LJC parameters or NULL.
 *   report_every : 0 = no diagnostics; R > 0 = FP64 diagnostics at steps
 *           0, R, 2R, ... <= nsteps, written as rows of 8 doubles
 *           (K, U, Px, Py, Pz, Lx, Ly, Lz) into diag (host or device,
 *           floor(nsteps / R) + 1 rows). The FP64 reductions are the only
 *           double-precision arithmetic on the GPU.
 *   trace : NULL, or (nsteps + 1) * n float4 receiving the positions x_0 ..
 *           x_nsteps (used by reverse-mode recomputation).
 *   state_lo : NULL, or 2 * n float4 holding the low parts of a two-float
 *           state (first n: x_lo, next n: v_lo; zero them to start). With it,
 *           every kick and drift is a compensated (TwoSum) update of
 *           (hi, lo), so FP32 rounding does not drift over many steps
 *           (Sec. 3.2: higher precision only where it is needed). Forces are
 *           always evaluated at the FP32 positions pos_m.
 * Host pointers are accepted as in nbody_forces (all of pos_m, vel, acc, prm
 * on the host); then the call synchronizes. A host diag also synchronizes.
 * Launches on the stream: for a packed tile one pair-interleave launch before
 * the first evaluation (with NBODY_ACC_VALID it also applies the first
 * half-kick and drift), then per evaluation the force kernel and one finalize
 * kernel, which kicks and drifts, adds the diagnostics of a report step and
 * writes the next evaluation's source copy; every launch after the first is a
 * programmatic dependent launch.
 * --------------------------------------------------------------------------- */
int nbody_step(void *pos_m, void *vel, void *acc, const void *prm, int64_t n, float dt,
               int32_t nsteps, int32_t report_every, double *diag, void *trace, void *state_lo,
               const nbody_params *params, nbody_stream_t stream);

/* ---------------------------------------------------------------------------
 * Batched ensembles (Sec. 3.4, small systems): many
 * independent systems of uneven size in one persistent launch per step.
 * System k occupies particles [offset, offset + n) of the shared arrays.
 * --------------------------------------------------------------------------- */
typedef struct {
    int64_t offset; /* first particle; a multiple of 4                        */
    int32_t n;      /* particles in the system, >= 1                          */
    int32_t law;    /* NBODY_LAW_*: gravity, LJC or LJC(linear) per system;
                       LJC systems read prm packed with their own kq          */
    float G;        /* gravity constant (gravity systems)                     */
    float eps2;     /* squared softening (gravity systems)                    */
    float dt;       /* leapfrog step of this system                           */
    int32_t reserved;
} nbody_system;

typedef struct nbody_batch_plan nbody_batch_plan;

/* Build the work list (longest items first) for a host table of systems.
 * flags: NBODY_PRECISE_RSQRT / NBODY_NO_COMPENSATION. tile = -1 picks the
 * tuned configuration. Allocates device memory; no stream work. */
int nbody_batch_plan_create(const nbody_system *systems, int32_t nsys, uint32_t flags,
                            int32_t tile, nbody_batch_plan **plan);
int nbody_batch_plan_destroy(nbody_batch_plan *plan);
/* Total particles covered by the plan (max offset + n). */
int64_t nbody_batch_plan_particles(const nbody_batch_plan *plan);

/* nsteps == 0: forces only (acc = a(x) of every system). nsteps > 0: nsteps
 * leapfrog steps per system (acc must hold a(x) on entry when ACC_VALID is set
 * in `flags`; otherwise it is computed first). With use_graph != 0 the whole
 * nsteps loop is captured once into a CUDA graph per (plan, nsteps, pointers)
 * and replayed. Device pointers only. */
int nbody_batch_run(nbody_batch_plan *plan, void *pos_m, void *vel, void *acc,
                    const void *prm, int32_t nsteps, uint32_t flags, int32_t use_graph,
                    nbody_stream_t stream);

/* One-shot convenience: plan, run, destroy (synchronizes the stream). The
 * system table is on the host. */
int nbody_forces_batched(const nbody_system *systems, int32_t nsys, void *pos_m, void *vel,
                         void *acc, const void *prm, int32_t nsteps, uint32_t flags,
                         nbody_stream_t stream);

/* ---------------------------------------------------------------------------
 * nbody_adjoint -- one vector-Jacobian product of the force law (derived from
 * Eq. 1 and Table 1 by differentiation; the paper has no adjoint):
 *   grad_x[k] (+)= alpha * sum_i (d a_i / d x_k)^T lam_i
 *   grad_m[k] (+)= alpha * sum_i lam_i . d a_i / d m_k
 *   grad_types (+)= alpha * (d/d sigma_t, d/d eps_t of sum_i lam_i . a_i),
 *                  2 * ntypes doubles (both LJC laws; NULL to skip)
 *   params->law : gravity, LJC or LJC(linear)
 *   pos_m, prm : as in nbody_forces; lam : n float4 (w ignored)
 *   grad_x : n float4 (w ignored on input, 0 on output); grad_m : n floats
 * With NBODY_ACCUMULATE the outputs are added to, else overwritten.
 * Device pointers only.
 * --------------------------------------------------------------------------- */
int nbody_adjoint(const void *pos_m, const void *prm, const void *lam, void *grad_x,
                  float *grad_m, double *grad_types, int32_t ntypes, float alpha, int64_t n,
                  const nbody_params *params, nbody_stream_t stream);

/* nbody_adjoint_leapfrog -- reverse of `k` leapfrog steps n = k-1 .. 0 over
 * stored positions xs[0..k-1] (k * n float4, as written by nbody_step's
 * trace), each reverse step being
 *   lam_v += dt * lam_x;   lam_x += w_n * J(x_n)^T lam_v
 * with w_n = dt, except w_0 = dt/2 when `first` is nonzero (the chunk starts
 * at step 0 of the trajectory). Mass and per-type gradients accumulate with
 * the same weights into grad_m / grad_types (which are NOT cleared).
 * lam_x, lam_v : n float4, in/out. Device pointers only.
 * --------------------------------------------------------------------------- */
int nbody_adjoint_leapfrog(const void *xs, const void *prm, int64_t n, int32_t k, float dt,
                           int32_t first, void *lam_x, void *lam_v, float *grad_m,
                           double *grad_types, int32_t ntypes, const nbody_params *params,
                           nbody_stream_t stream);

/* ---------------------------------------------------------------------------
 * Tile configurations and tuning.
 * --------------------------------------------------------------------------- */
/* Number of compiled tile configurations for tile table `law` (0 gravity,
 * 1 LJC, 2 LJC linear, 3 the mixed-law batched kernel, 4 gravity with
 * fixed-point accumulation, 5 the gravity VJP, 6 the LJC VJP, 7 acceleration
 * + jerk, 8 the LJC(linear) VJP), or a negative status. */
int nbody_tile_count(int32_t law);
/* Kind bits of a tile configuration (nbody_tile_info). */
enum {
    NBODY_TILE_PACKED = 1,     /* reads pair-interleaved sources: a force evaluation
                                  is preceded by one interleave launch (within an
                                  nbody_step call, only the first) */
    NBODY_TILE_SYMMETRIC = 2,  /* Newton-symmetric block pairs: each unordered pair
                                  evaluated once and applied to both particles; j_tile
                                  is the block size; for the force laws and the
                                  gravity VJP the j-split
                                  cuts each block's sources into 1, 2, 4 or 8 parts
                                  (one CTA each; 0: one part, other values rounded
                                  down). Softened gravity (eps2 > 0, without
                                  NBODY_NO_COMPENSATION) adds each block's partial
                                  sums as fixed point with integer atomics (an
                                  integer part and a 2^-32 fraction word per
                                  component: every FP32 partial is added exactly,
                                  whatever the softening; Sec. 3.2, the GRAPE-6
                                  scheme; bitwise reproducible) into 64 bytes of
                                  scratch per particle; the
                                  other cases keep one partial per particle and
                                  block, so the tile is refused (explicit tile) or
                                  replaced by the default tile (tuned) when those
                                  partials would exceed an eighth of the device's
                                  memory or 16 GiB. Never used for subsets or by
                                  the allocation-free entry point */
};
/* Describe configuration `tile` of `law`: threads per CTA (consumer warps),
 * i-particles per thread, j-lanes per warp, j-tile length, and its kind
 * (NBODY_TILE_* bits; 0: a one-sided kernel reading pos_m/prm directly). Any
 * output pointer may be NULL. */
int nbody_tile_info(int32_t law, int32_t tile, int32_t *threads, int32_t *i_per_thread,
                    int32_t *j_lanes, int32_t *j_tile, int32_t *kind);
/* Install the tuned (tile, jsplit) for (tile table law, n-bucket); bucket =
 * floor(log2 n) (the batched table uses bucket 0). Used by params->tile == -1. */
int nbody_set_tuned(int32_t law, int32_t log2n, int32_t tile, int32_t jsplit);
/* Query the configuration a call with (law, n) and tile == -1 would use. */
int nbody_get_config(int32_t law, int64_t n, int32_t *tile, int32_t *jsplit);
/* Device scratch bytes a call of nbody_forces / nbody_step with these params
 * and n requests from the library's per-(device, stream) workspace: the
 * pair-interleaved source copy of packed tiles, the per-slice partial sums and
 * (nbody_step with report_every) `report_rows` rows of diagnostics. The arena
 * grows to the largest request and is reused; a call made while a stream is
 * being captured into a CUDA graph must not need more than that stream already
 * holds (run it once uncaptured first). Needs the device (the j-split depends
 * on its SM count). The paper has no counterpart (it keeps everything in GPU
 * textures). */
int nbody_workspace_size(const nbody_params *params, int64_t n, int32_t report_rows,
                         size_t *bytes);
/* Autotune tile table `table` at size n on the caller's device inputs (the
 * paper tunes its unrolling by hand, Sec. 3.3; this searches the compiled
 * configurations instead). Every tile x j-split in {0 (auto), 1, 2, 4, 8, 16,
 * 32} that fits n (Newton-symmetric tiles: the splits their plan takes, and only
 * where their partial-sum cap admits n) is run once to warm up and `reps` (1..1000) more times, timed
 * with CUDA events on `stream`; the median decides. The fastest is installed
 * with nbody_set_tuned for bucket floor(log2 n) and returned in best_tile,
 * best_jsplit and best_ms (milliseconds per call; any may be NULL). What is
 * timed: tables 0-2 nbody_forces (law = table), 4 nbody_forces with
 * NBODY_FIXED_POINT (eps2 > 0), 5 / 6 / 8 nbody_adjoint (gravity / LJC / LJC
 * linear, with lambda = pos_m), 7 nbody_forces_jerk (velocities = pos_m); G = 1,
 * softening eps2. prm: the LJC parameters for tables 1, 2, 6 and 8, else
 * ignored. Outputs
 * go to library scratch. Table 3 (batched) returns NBODY_EUNSUPPORTED: the
 * package tunes it over a system table. Synchronizes `stream`; on any error
 * nothing is installed. */
int nbody_tune(int32_t table, const void *pos_m, const void *prm, int64_t n, float eps2,
               int32_t reps, int32_t *best_tile, int32_t *best_jsplit, float *best_ms,
               nbody_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* NBODY_H */
