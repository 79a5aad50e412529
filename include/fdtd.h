/*
 * fdtd.h - C ABI of the GB300 (sm_103a) Yee FDTD library (libfdtd.so).
 *
 * The library advances Maxwell's curl equations (J = 0) on a perfectly
 * conducting (PEC) box cavity with the Yee leapfrog scheme of He, Andersson and
 * Markidis, "Optimizing FDTD Solvers for Electromagnetics: A Compiler-Guided
 * Approach with High-Level Tensor Abstractions" (arXiv 2504.09118):
 *   Sec. 2, Eq. 1   - the curl equations;
 *   Sec. 2, Eq. 2   - the staggered update of the six components;
 *   Sec. 2.1, Listing 1 - one step = H from curl E, boundary, E from curl H, boundary;
 *   Sec. 4          - the benchmark workload: a PEC cavity from a random state;
 *   Sec. 6          - higher-order schemes (fdtd_set_order: the fourth-order differences).
 *
 * Units and conventions
 *   nx, ny, nz are cell counts; dx = dy = dz = dx.  State after n steps is
 *   (H^{n-1/2}, E^n).  One step:
 *     H -= ch * curl E   (all H in their Yee extent; normal H on a face is unchanged)
 *     E += ce * curl H   (E tangential to a face stays exactly 0: PEC)
 *   ce = dt/(eps*dx) at each E position, ch = dt/(mu*dx) at each H position.
 *
 * Canonical layout (every field and coefficient array crossing this ABI)
 *   float[(nz+1)*(ny+1)*(nx+1)], C order, x fastest: element (i,j,k) is at
 *   ((k*(ny+1) + j)*(nx+1) + i).  Component c at (i,j,k) sits at its Yee position
 *     Ex (i+1/2, j, k)     i<nx,  j<=ny, k<=nz
 *     Ey (i, j+1/2, k)     i<=nx, j<ny,  k<=nz
 *     Ez (i, j, k+1/2)     i<=nx, j<=ny, k<nz
 *     Hx (i, j+1/2, k+1/2) i<=nx, j<ny,  k<nz
 *     Hy (i+1/2, j, k+1/2) i<nx,  j<=ny, k<nz
 *     Hz (i+1/2, j+1/2, k) i<nx,  j<ny,  k<=nz
 *   Entries outside a component's extent are ignored on input and written 0
 *   on output.  Field arrays are passed as f[6] = {Ex, Ey, Ez, Hx, Hy, Hz}.
 *
 * Errors: every int-returning call returns FDTD_OK (0) or a negative status
 * and never aborts.  The main calls mark their extent with NVTX ranges named after them (visible to
 * Nsight tools; no cost without one).  A failed call leaves a message in fdtd_last_error(ctx).
 * Device-side errors (a bounded wait that ran out) are latched in a device
 * status word and reported by the next call that synchronises the stream.
 *
 * Threading: a context (or batch) must not be used from two host threads at once.
 */
#ifndef FDTD_H
#define FDTD_H

#if defined(__GNUC__)
#define FDTD_API __attribute__((visibility("default")))
#else
#define FDTD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fdtd_ctx fdtd_ctx;
typedef struct fdtd_batch fdtd_batch;

/* Storage precision of the fields in device memory.  Arithmetic is always FP32;
 * FP16/BF16 store E scaled by a power of two s_E and H by s_H, chosen at
 * fdtd_set_fields (s = 2^(8 - ceil(log2 max|F|)) over the three components of
 * the field), rounded to nearest even. */
enum fdtd_storage { FDTD_F32 = 0, FDTD_F16 = 1, FDTD_BF16 = 2 };

enum fdtd_status {
    FDTD_OK = 0,
    FDTD_ERR_ARG = -1,       /* invalid argument (NULL, size, enum, mismatched batch member) */
    FDTD_ERR_OOM = -2,       /* device allocation failed */
    FDTD_ERR_CUDA = -3,      /* a CUDA runtime/driver call failed */
    FDTD_ERR_TIMEOUT = -4,   /* a kernel's bounded wait ran out; fields of that step are undefined */
    FDTD_ERR_STATE = -5,     /* call not valid in the current state (e.g. step before set_fields) */
    FDTD_ERR_UNSTABLE = -6   /* Courant bound violated: max sqrt(3 ce ch) > 1 */
};

/* Step kernels (fdtd_tuning.kernel). */
enum fdtd_kernel {
    FDTD_KERNEL_AUTO = 0,    /* TEMPORAL with 16-row tiles where it applies (else FUSED; SIMPLE for
                                per-position coefficient arrays); fdtd_autotune picks by timing */
    FDTD_KERNEL_SIMPLE = 1,  /* two launches per step (H, then E), one thread per cell; unfused baseline */
    FDTD_KERNEL_FUSED = 2,   /* one TMA-pipelined launch per step: H then E fused in a z-march */
    FDTD_KERNEL_TEMPORAL = 3, /* two steps per launch (temporal blocking); an odd count ends with one FUSED step */
    FDTD_KERNEL_TEMPORAL2 = 4, /* TEMPORAL with two tile rows per consumer warp (tile_y 12 or 16): same tiles and
                                 results (FP32: bit for bit), fewer instructions per cell-step */
    FDTD_KERNEL_TEMPORAL3 = 5 /* three steps per launch (single cavities, second order; tile_y 8, 10 or 12; 58-column
                                 tiles); a remainder ends with FUSED steps; FP32 results bit for bit those of
                                 TEMPORAL */
};

/* Launch configuration of the step kernel; zero fields take the default. */
typedef struct fdtd_tuning {
    int kernel;       /* enum fdtd_kernel */
    int tile_y;       /* fused: cells per tile along y (FUSED: 4, 8 or 16, fourth order also 12; TEMPORAL:
                         8, 12 or 16; TEMPORAL2: 12 or 16; TEMPORAL3: 8, 10 or 12; AUTO: any of these,
                         each kernel taking its default when the value is not one of its own); x tile is
                         64 cells (TEMPORAL, TEMPORAL2: 60; TEMPORAL3: 58) */
    int zchunk;       /* fused: planes per tile along z (>= 1); 0 = choose for load balance */
    int ctas_per_sm;  /* fused: persistent CTAs per SM (1 or 2); 0 = as many as fit */
    int stages;       /* fused: TMA pipeline depth in planes (3..8, lowered to fit shared memory); 0 = default */
    int use_graph;    /* 1 = replay fdtd_step / fdtd_batch_step through a captured CUDA graph */
} fdtd_tuning;

/*
 * fdtd_create - allocate a cavity of nx*ny*nz cells on the current device.
 * Defines the grid and coefficients of Sec. 2, Eq. 2: ce = dt/(eps dx) multiplies curl H in the E
 * update, ch = dt/(mu dx) multiplies curl E in the H update; the box walls are PEC as in the
 * benchmark cavity of Sec. 4.
 *   dt, dx      time step and cell size (> 0).
 *   ce[3]       host canonical arrays of dt/(eps*dx) at the Ex, Ey, Ez
 *               positions, or NULL for vacuum (dt/dx everywhere).
 *   ch[3]       host canonical arrays of dt/(mu*dx) at the Hx, Hy, Hz
 *               positions, or NULL for vacuum.
 *   storage     enum fdtd_storage.
 *   cuda_stream cudaStream_t to issue all work on (NULL = legacy default stream).
 * The library copies the coefficients (compressing them to a one-byte material
 * id per cell plus a table when at most 256 distinct per-cell tuples occur)
 * and owns all device memory until fdtd_destroy.  With at most 31 tuples it
 * also keeps a second one-byte id per cell for the two-step kernels, which
 * codes the PEC faces the cell lies on (Sec. 2: tangential E vanishes on the
 * walls) into its table entry.  Fields start at zero.
 * Returns FDTD_ERR_UNSTABLE (and no context) when some cell has
 * sqrt(3 * ce * ch) > 1 for a co-located pair, FDTD_ERR_ARG for sizes < 1 or
 * > 32768 or non-positive coefficients.  On error *out is NULL.
 */
FDTD_API int fdtd_create(fdtd_ctx **out, int nx, int ny, int nz, double dt, double dx,
                const float *const ce[3], const float *const ch[3], int storage, void *cuda_stream);

/*
 * fdtd_set_fields - load the state (H^{n-1/2}, E^n) and reset the step counter.
 * The six staggered components of Sec. 2, Eq. 2 at their Yee positions; H is taken half a step
 * behind E because a step of Sec. 2.1, Listing 1 updates H first (Eq. 2 labels the same state
 * (E^{n+1/2}, H^{n+1}); the two labellings differ only by a half-step shift of the clock).
 *   f[6]       canonical FP32 arrays; host pointers when on_device == 0, CUDA
 *              device pointers when on_device == 1.  Read during the call only, on the
 *              context's stream: device data written on another stream must be complete
 *              before the call (the Python binding synchronises torch's current stream).
 * Tangential E on the faces is written as 0 whatever the input holds.
 * Synchronises the stream before returning.
 */
FDTD_API int fdtd_set_fields(fdtd_ctx *ctx, const float *const f[6], int on_device);

/* fdtd_prefetch_fields - start copying the next fields from host memory while the context computes.
 * f[6]: host arrays, canonical layout as fdtd_set_fields (page-locked memory for the copy to overlap
 * the context's kernels: pageable memory is copied but not overlapped).  The six arrays are copied into
 * a device area owned by the context (6 x (nx+1)(ny+1)(nz+1) floats, allocated at the first call) on a
 * second stream; the call returns without waiting.  They must stay valid and unchanged until the
 * matching fdtd_set_fields_prefetched returns.  FDTD_ERR_STATE while an earlier prefetch has not been
 * loaded.  Lets a caller overlap the host-to-device load of its next solve with the current one. */
FDTD_API int fdtd_prefetch_fields(fdtd_ctx *ctx, const float *const f[6]);

/* fdtd_set_fields_prefetched - fdtd_set_fields from the arrays of the last fdtd_prefetch_fields (waits
 * for their copy on the GPU, not on the host, then loads them as fdtd_set_fields does from device
 * arrays).  FDTD_ERR_STATE when no prefetch is pending or the context is a batch member. */
FDTD_API int fdtd_set_fields_prefetched(fdtd_ctx *ctx);

/*
 * fdtd_step - advance nsteps >= 0 leapfrog steps, asynchronously on the context's stream.
 * One step is Sec. 2.1, Listing 1: the H update of Sec. 2, Eq. 2 (H -= ch curl E, with the minus
 * sign of Faraday's law), the H boundary handling (nothing to do on a PEC box: normal H on a face
 * sees zero curl), the E update of Eq. 2 (E += ce curl H), the E boundary handling (tangential E
 * on the faces stays 0).  Results equal those of that sequence up to FP32 rounding order.  Launch errors are returned here; device-side errors
 * at the next synchronising call.
 */
FDTD_API int fdtd_step(fdtd_ctx *ctx, int nsteps);

/*
 * fdtd_get_fields - the state (H^{n-1/2}, E^n) of Sec. 2, Eq. 2 after the steps taken,
 * written into f[6] (canonical FP32; host or
 * device pointers as on_device says; device buffers are written on the context's
 * stream, so other streams must be done with them).  Entries outside each extent are 0.
 * Synchronises the stream; returns a latched device error if one occurred.
 */
FDTD_API int fdtd_get_fields(fdtd_ctx *ctx, float *const f[6], int on_device);

/*
 * fdtd_energy - discrete Yee energy of the current state, accumulated in FP64:
 *   W^n = 1/2 sum eps |E^n|^2 + 1/2 sum mu H^{n-1/2} . H^{n+1/2},
 *   eps = dt/(ce dx), mu = dt/(ch dx), cell volume 1, with H^{n+1/2} formed on the
 *   fly.  It is the invariant of the Eq. 2 leapfrog on a lossless PEC cavity.
 * The paper defines no energy: this is the quadratic form the leapfrog conserves exactly (the
 * plain 1/2 sum eps E^2 + mu H^2 with both at one time level is not conserved), chosen as the
 * check of a lossless run.  Every term is formed and summed in FP64 from the stored values.
 * Synchronises the stream.
 */
FDTD_API int fdtd_energy(fdtd_ctx *ctx, double *W);

/*
 * fdtd_divergence - L2 norms (FP64) of the discrete divergences:
 *   divE at interior nodes: sum_c E_c/ce_c (node) - E_c/ce_c (node - e_c);
 *   divH at every cell:     sum_c H_c/ch_c (cell + e_c) - H_c/ch_c (cell).
 * Both are invariant under exact Yee stepping (the discrete divergence of a discrete curl is
 * zero).  The paper defines neither; they are the second invariant checked on a lossless run.
 * Every term is formed and summed in FP64 from the stored values.  Synchronises the stream.
 */
FDTD_API int fdtd_divergence(fdtd_ctx *ctx, double *divE_l2, double *divH_l2);

/* fdtd_sync - wait for the context's stream; returns a latched device error, if any. */
FDTD_API int fdtd_sync(fdtd_ctx *ctx);

/* fdtd_set_tuning - choose the step kernel and its launch shape (NULL = defaults).  With spatial
 * order 4 (fdtd_set_order) the kernels TEMPORAL, TEMPORAL2 and TEMPORAL3 and stages = 3 are FDTD_ERR_ARG;
 * so is a tile_y the chosen kernel does not take. */
FDTD_API int fdtd_set_tuning(fdtd_ctx *ctx, const fdtd_tuning *t);

/*
 * fdtd_set_order - spatial order of the curl differences: 2 (Eq. 2; the default) or 4.
 *
 * Sec. 6 names higher-order schemes as the way to raise FDTD's arithmetic intensity; order 4 is the
 * staggered fourth-order (2,4) scheme: every difference f(p+1/2) - f(p-1/2) of Eq. 2 becomes
 *   c1 [f(p+1/2) - f(p-1/2)] + c2 [f(p+3/2) - f(p-3/2)],   c1 = 9/8, c2 = -1/24,
 * with the PEC walls closed by image theory (about each wall tangential E is odd and tangential H
 * even; a tap one position past a wall reads that image).  Time stepping, layout, PEC (tangential E
 * stays 0, normal H constant) and currents are unchanged.  fdtd_energy and fdtd_divergence then use
 * the same differences (the energy W^n with the fourth-order curl, the divergences with D = E/ce
 * mirrored evenly and B = H/ch oddly past a wall), the invariants of this scheme.
 *
 * Kernels with order 4: FUSED (and AUTO) run the fused fourth-order kernel (one launch per step;
 * tile_y 4, 8, 12 or 16, default 12; stages 4..8, default the deepest ring that fits), SIMPLE the unfused one (also the path for per-position
 * coefficient arrays); TEMPORAL is not available.  Returns FDTD_ERR_UNSTABLE when the scheme's
 * Courant bound fails (order 4: max sqrt(3 ce ch) * 7/6 > 1, as the difference's symbol reaches
 * c1 - c2 = 7/6), FDTD_ERR_ARG for another order or a TEMPORAL / stages = 3 tuning, FDTD_ERR_STATE
 * for a batch member (fourth-order contexts are not batched).  Applies from the next call on;
 * synchronises the stream.
 */
FDTD_API int fdtd_set_order(fdtd_ctx *ctx, int order);

/* fdtd_get_order - the context's spatial order (2 or 4), -1 for NULL. */
FDTD_API int fdtd_get_order(const fdtd_ctx *ctx);

/* fdtd_autotune - choose the step kernel and launch shape by timing candidates on this
 * context's own state: the one-step kernel with 4, 8, 16-row tiles, the two-step kernel with
 * 8, 12, 16-row tiles and 4 or 6 ring slots, the three-step kernel with 8, 10, 12-row tiles, and the
 * two-step kernel with two rows per warp with 12 and 16-row tiles (graphs on).  Each candidate runs trial_steps steps
 * (rounded up to a multiple of 16; <= 0: 16) after one untimed run of the same length, timed
 * with CUDA events on the context's stream.  The fields are copied aside first (one extra copy
 * of the active arrays, freed before return) and restored afterwards, so the state and
 * fdtd_steps_done are unchanged.  The choice is kept per (nx, ny, nz, storage, coefficient
 * kind, spatial order) for the life of the process: a later call for the same shape applies it
 * without trials.  Contexts with per-position coefficient arrays keep the unfused kernel; with
 * order 4 the candidates are the fused fourth-order kernel with 4, 8, 12, 16-row tiles and the
 * deepest ring that fits or 4 slots.  out
 * (may be NULL) receives the chosen tuning, ms_per_step (may be NULL) its time per step.
 * Requires fdtd_set_fields; synchronises the stream. */
FDTD_API int fdtd_autotune(fdtd_ctx *ctx, int trial_steps, fdtd_tuning *out, double *ms_per_step);

/* fdtd_set_sources - point currents, the J of Sec. 2, Eq. 1 (the benchmark's J = 0): in the step
 * from E^n to E^{n+1} (n counted from the last fdtd_set_fields) the E update also subtracts
 *   ce_c(i,j,k) * dx * wave[s * wave_len + n]          (0 once n >= wave_len)
 * at source s: component comp[s] (0 Ex, 1 Ey, 2 Ez) at canonical index ijk[3s..3s+2], which must be
 * an E position inside the cavity and not tangential to a face (ERR_ARG otherwise).  Sources at the
 * same position add up.  nsrc = 0 removes them.  All arrays are host memory, copied.  While currents
 * or probes are set, steps run the one-step kernel followed by one small launch for them (the
 * two-step kernel has no point between its steps where J could enter).  Synchronises the stream. */
FDTD_API int fdtd_set_sources(fdtd_ctx *ctx, int nsrc, const int *comp, const int *ijk, const float *wave,
                              int wave_len);

/* fdtd_set_probes - after every step, record component comp[p] (0..5 = Ex..Hz; an H value is
 * H^{n+1/2}) at canonical index ijk[3p..3p+2] (0 <= i < nx, 0 <= j < ny, 0 <= k < nz), in physical
 * units, into a device buffer of `capacity` steps starting with the next step; samples beyond the
 * capacity are dropped.  nprobe = 0 removes them.  fdtd_set_fields restarts the recording.
 * Synchronises the stream. */
FDTD_API int fdtd_set_probes(fdtd_ctx *ctx, int nprobe, const int *comp, const int *ijk, int capacity);

/* fdtd_get_probes - copy the probe buffer to host memory out[nprobe * capacity] (probe-major:
 * out[p * capacity + n] is probe p after the n-th recorded step) and the number of recorded steps.
 * Synchronises the stream. */
FDTD_API int fdtd_get_probes(fdtd_ctx *ctx, float *out, int *nrecorded);

/* fdtd_steps_done - steps taken since the last fdtd_set_fields (-1 for a NULL ctx). */
FDTD_API long long fdtd_steps_done(const fdtd_ctx *ctx);

/* fdtd_device_bytes - device memory the context holds (fields, ping-pong copy, coefficients, material ids). */
FDTD_API long long fdtd_device_bytes(const fdtd_ctx *ctx);

/* fdtd_destroy - free the context and its device memory (synchronises first). NULL is a no-op. */
FDTD_API void fdtd_destroy(fdtd_ctx *ctx);

/* fdtd_last_error - message of the last failed call on ctx (or of the last
 * failed fdtd_create when ctx is NULL); valid until the next call on ctx. */
FDTD_API const char *fdtd_last_error(const fdtd_ctx *ctx);

/* ------------------------------------------------------------------------
 * Batches: many independent cavities advanced by one persistent launch per
 * step over a packed list of equal-size tiles (all members must share the
 * storage precision and stream).  A member keeps its own fields; adding or
 * removing members between steps is allowed (continuous batching).
 * ------------------------------------------------------------------------ */

/* fdtd_batch_create - empty batch for members of the given storage, on cuda_stream. */
FDTD_API int fdtd_batch_create(fdtd_batch **out, int storage, void *cuda_stream);

/* fdtd_batch_add - add a cavity (after its fdtd_set_fields); it keeps its state.  The cavity may
 * use its own stream: fdtd_batch_remove orders that stream after the batch's work. */
FDTD_API int fdtd_batch_add(fdtd_batch *b, fdtd_ctx *ctx);

/* fdtd_batch_remove - remove a member; it can be stepped or read on its own afterwards.  Does not
 * wait for the GPU: the member's stream is made to wait for the batch work enqueued so far.
 * The member's fdtd_steps_done is brought up to date here. */
FDTD_API int fdtd_batch_remove(fdtd_batch *b, fdtd_ctx *ctx);

/* fdtd_batch_set_steps - the member takes exactly nsteps more steps of this batch and is then
 * skipped by every later launch (its state frozen) until it is removed.  Lets members with
 * different step counts share launches without stopping the batch for each of them. */
FDTD_API int fdtd_batch_set_steps(fdtd_batch *b, fdtd_ctx *ctx, long long nsteps);

/* fdtd_batch_steps_done - the batch's step clock: steps enqueued since the batch was created
 * (-1 for NULL).  A member added at clock c with fdtd_batch_set_steps(n) is done at clock c + n. */
FDTD_API long long fdtd_batch_steps_done(const fdtd_batch *b);

/* fdtd_batch_step - advance every member nsteps steps, asynchronously on the batch stream.  With
 * the TEMPORAL kernel each launch takes two steps; a member with one step left (its own count, or
 * an odd nsteps) takes it in the same launch and stores its one-step result, so every member's
 * result is bit-identical to stepping it alone with FP32 storage. */
FDTD_API int fdtd_batch_step(fdtd_batch *b, int nsteps);

/* fdtd_batch_set_tuning - launch shape for the batch kernel: FUSED (one step per launch) or TEMPORAL,
 * TEMPORAL2 or AUTO (two steps per launch; TEMPORAL3 is for single cavities: FDTD_ERR_ARG); may change
 * between fdtd_batch_step calls.  With one CTA per SM and every running member stopping at the same
 * clock, tiles are assigned to the CTAs on the host for balance; otherwise they are dealt round-robin. */
FDTD_API int fdtd_batch_set_tuning(fdtd_batch *b, const fdtd_tuning *t);

/* fdtd_batch_autotune - fdtd_autotune for a batch over its current members: the one-step kernel
 * with 4, 8, 16-row tiles and the two-step kernels with 8, 12, 16-row tiles (two rows per warp:
 * 12, 16), each timed over
 * trial_steps batch steps (rounded up to a multiple of 16; <= 0: 16) after an untimed run.
 * Members' fields, step counts and the batch clock are restored afterwards.  Not cached (the
 * members change).  out / ms_per_step may be NULL.  Synchronises the batch stream. */
FDTD_API int fdtd_batch_autotune(fdtd_batch *b, int trial_steps, fdtd_tuning *out, double *ms_per_step);

/* fdtd_batch_retune - online re-tuning from a size-bucket model, for a batch whose members change
 * (continuous batching).  The bucket of a batch is (storage, floor(log2 C)) with C the total cell
 * count of its running members (those with steps left; all members when none has).
 * The first call for a bucket runs fdtd_batch_autotune on the batch as it is (same trials, same state
 * restoration) and keeps the choice for the life of the process; a later call whose batch falls in a
 * bucket already timed applies that choice without trials (and without touching the batch when the
 * choice is the current tuning).  out / ms_per_step (the bucket's timed ms per step) / timed (1 when
 * this call ran the trials, 0 when it used the model) may be NULL.  Errors as fdtd_batch_autotune;
 * synchronises the batch stream only when it times. */
FDTD_API int fdtd_batch_retune(fdtd_batch *b, int trial_steps, fdtd_tuning *out, double *ms_per_step, int *timed);

/* fdtd_batch_size - number of members (-1 for NULL). */
FDTD_API int fdtd_batch_size(const fdtd_batch *b);

/* fdtd_batch_sync - wait for the batch stream; returns a latched device error, if any. */
FDTD_API int fdtd_batch_sync(fdtd_batch *b);

/* fdtd_batch_destroy - release the batch (members are not destroyed). */
FDTD_API void fdtd_batch_destroy(fdtd_batch *b);

/* fdtd_batch_last_error - message of the last failed batch call. */
FDTD_API const char *fdtd_batch_last_error(const fdtd_batch *b);

/* ------------------------------------------------------------------------
 * z-slab decomposition of one cavity (domain decomposition; Sec. 6 names it among the ways FDTD is
 * spread over many processors).  A slab context owns the cells of global planes [k0, k1) of an
 * nx*ny*nz_global cavity and keeps `ghost` copies of its neighbours' cells on each side that has a
 * neighbour.  Steps run the ordinary kernels on the slab alone: on a ghost side the slab's local
 * boundary acts as a PEC wall, which is wrong there, and the error moves inwards by the reach of
 * the differences per step (1 plane for Eq. 2, 3 for order 4).  So after the ghost cells are
 * refreshed from the neighbours' owned cells, the owned cells stay exact for floor(ghost / reach)
 * steps; fdtd_step returns FDTD_ERR_STATE for more.  The owned values are then bit-identical to
 * the same cells of the undivided cavity (FP32 storage; 16-bit storage as well when every slab
 * stores with the same scales, see fdtd_set_storage_scales).
 * ------------------------------------------------------------------------ */

/* fdtd_create_slab - the slab [k0, k1) of an nx*ny*nz_global cavity, with g_lo = (k0 > 0 ? ghost : 0)
 * ghost cells below and g_hi = (k1 < nz_global ? ghost : 0) above.  It is a context of
 * nz_local = k1 - k0 + g_lo + g_hi cells along z whose local plane p is global plane k0 - g_lo + p;
 * ce / ch are host canonical arrays of those local planes (as for fdtd_create with nz = nz_local; NULL
 * for vacuum), storage and stream as for fdtd_create.  Every other call (set/get fields, step, order,
 * tuning) applies to the slab as to a cavity of nz_local cells.  A load leaves the ghost cells
 * untrusted: import (or exchange) both ghost sides before the first step.  FDTD_ERR_ARG when
 * [k0, k1) is empty or outside [0, nz_global), ghost is not in [1, 64], the ghosts would reach outside
 * the cavity, or a slab with a neighbour owns fewer than `ghost` planes. */
FDTD_API int fdtd_create_slab(fdtd_ctx **out, int nx, int ny, int nz_global, int k0, int k1, int ghost, double dt,
                              double dx, const float *const ce[3], const float *const ch[3], int storage,
                              void *cuda_stream);

/* fdtd_slab_info - info[7] = {nz_global, k0, k1, g_lo, g_hi, ghost, steps the owned cells stay exact
 * before the next exchange (INT_MAX for a slab without neighbours)}.  FDTD_ERR_STATE for a context not
 * made by fdtd_create_slab. */
FDTD_API int fdtd_slab_info(const fdtd_ctx *ctx, int info[7]);

/* fdtd_slab_halo_bytes - bytes that fdtd_slab_export writes and fdtd_slab_import reads for one side:
 * 6 fields x ghost planes x ny x pitch storage elements (pitch = nx rounded up to 32; 4 or 2 bytes per
 * element).  -1 for NULL or a context that is not a slab. */
FDTD_API long long fdtd_slab_halo_bytes(const fdtd_ctx *ctx);

/* fdtd_slab_export - copy the owned boundary cells of one side (side 0: the `ghost` lowest owned planes,
 * 1: the highest) into buf, laid out as [field Ex..Hz][plane][y][x with the padded pitch] in the storage
 * type and scaling of the slab (fdtd_slab_halo_bytes bytes).  on_device = 1: buf is device memory and
 * the copy is ordered on the slab's stream (asynchronous); 0: host memory, the call waits for it.  The
 * neighbour on that side imports the buffer.  FDTD_ERR_ARG for a side that is a wall of the cavity. */
FDTD_API int fdtd_slab_export(fdtd_ctx *ctx, int side, void *buf, int on_device);

/* fdtd_slab_import - write a neighbour's export into the ghost cells of one side (0 below, 1 above) and
 * restore that side's step allowance.  The exporting slab must have the same nx, ny, storage, ghost
 * depth and storage scales, and its state must be at the same step.  Stream ordering as export. */
FDTD_API int fdtd_slab_import(fdtd_ctx *ctx, int side, const void *buf, int on_device);

/* fdtd_slab_exchange - both directions between two neighbouring slabs (lo's k1 == hi's k0), device to
 * device (the same GPU, or two GPUs through unified addressing): lo's highest owned cells into hi's
 * lower ghosts and hi's lowest owned cells into lo's upper ghosts.  The copies run on lo's stream after
 * the work already enqueued on hi's stream, and hi's stream waits for them; no host synchronisation.
 * FDTD_ERR_ARG for slabs that are not neighbours or differ in size, storage, ghost depth or scales. */
FDTD_API int fdtd_slab_exchange(fdtd_ctx *lo, fdtd_ctx *hi);

/* fdtd_slab_energy - the part of the energy W (as fdtd_energy, FP64) that lies in the owned cells (the far
 * z face with the slab that has it); the energies of all slabs add up to the cavity's.  The ghost cells
 * must be current (no step since the last exchange on both sides), else FDTD_ERR_STATE.  Synchronises. */
FDTD_API int fdtd_slab_energy(fdtd_ctx *ctx, double *W);

/* fdtd_slab_divergence_sq - the owned parts of the squared divergence norms of fdtd_divergence (sums of
 * squares: add them over slabs, then take the square roots).  Conditions as fdtd_slab_energy. */
FDTD_API int fdtd_slab_divergence_sq(fdtd_ctx *ctx, double *divE2, double *divH2);

/* fdtd_set_storage_scales - fix the power-of-two scales s_E, s_H with which later loads store 16-bit fields
 * (0: chosen from the loaded data, the default).  Slabs of one cavity must share them: take
 * fdtd_storage_scale_of of the largest |E| and |H| of the whole cavity.  FDTD_ERR_ARG for a value that is
 * neither 0 nor a power of two, and from the next fdtd_set_fields when a loaded field times its fixed
 * scale exceeds the FP16 range.  Applies from the next fdtd_set_fields; no effect with FP32 storage. */
FDTD_API int fdtd_set_storage_scales(fdtd_ctx *ctx, double s_e, double s_h);

/* fdtd_storage_scale_of - the scale a load chooses for a field whose largest magnitude is maxabs:
 * 2^(8 - ceil(log2 maxabs)), 1 for maxabs <= 0 or not finite. */
FDTD_API double fdtd_storage_scale_of(double maxabs);

/* ------------------------------------------------------------------------
 * Diagnostics
 * ------------------------------------------------------------------------ */

/* fdtd_debug_inject_timeout - make the next fused step's first TMA stage never
 * be issued so that its bounded wait runs out after about limit_us microseconds;
 * the step then returns FDTD_ERR_TIMEOUT at the next synchronising call and the
 * context stays usable (its fields are undefined until the next set_fields).
 * Fault injection on the host side of a wait: no GPU fault is involved. */
FDTD_API int fdtd_debug_inject_timeout(fdtd_ctx *ctx, int limit_us);

/* fdtd_debug_fail_alloc - host-side fault injection for allocation failures: after `after` further
 * successful device allocations by the library (any context or batch), the next one fails once as if
 * the device were out of memory (the call that made it returns FDTD_ERR_OOM and releases what it had
 * taken); after < 0 disarms.  No GPU fault is involved.  Process-wide. */
FDTD_API int fdtd_debug_fail_alloc(int after);

/* fdtd_debug_tile_plan - host only (no GPU, no context): the work split that the fused kernels use for
 * one cavity with one persistent CTA per SM.  The cavity is cut into `cols` columns (x-y tiles) over nz
 * planes; a tile is a column over a z-chunk and costs (chunk length + prologue) plane-times, prologue
 * being the planes that prime the z recurrence (1 for the one-step kernel, 3 for the two-step kernel,
 * 4 for the fourth-order kernel).  zchunk > 0 fixes the chunk length (the last chunk takes the rest);
 * zchunk = 0 picks, among n equal chunks (n = 1..64) and n chunks of one length followed by the rest in
 * 1-4 pieces, the plan with the shortest makespan of greedy list scheduling over min(ctas, cols * nz)
 * CTAs.  Tiles are listed chunk-major, columns in order within a chunk, and each goes to the CTA that
 * becomes free first (lowest index on ties).
 *   chunks[0 .. *nchunks)  chunk lengths in z order (capacity max_chunks, caller-owned)
 *   *makespan              plane-times of the busiest CTA
 *   cta_of_tile            NULL, or *nchunks * cols entries (caller-owned): the CTA of each listed tile
 * Returns FDTD_ERR_ARG for non-positive sizes, a negative prologue or zchunk, a capacity below the
 * plan's chunk count, or more than 2^26 tiles with cta_of_tile given. */
FDTD_API int fdtd_debug_tile_plan(long long cols, int nz, int ctas, int prologue, int zchunk, int *chunks,
                                  int max_chunks, int *nchunks, long long *makespan, int *cta_of_tile);

/* fdtd_debug_pec_code, fdtd_debug_pec_table - host only (no GPU, no context): the PEC-coded material
 * ids that the two-step kernels read for contexts with 1 <= ntab <= 31 material tuples.  Tangential E
 * vanishes on the PEC walls (Sec. 2); these write that condition as materials, so that the kernels'
 * inner loop applies no per-cell masks.
 *   fdtd_debug_pec_code   *code = the coded id of a cell of material id (0 <= id < ntab) at cell
 *                         (i, j, k), i, j, k >= 0: 1 + id + ntab x faces, where faces has bit 0 set
 *                         for i = 0, bit 1 for j = 0 and bit 2 for k = 0.  Cells outside the cavity
 *                         read code 0.
 *   fdtd_debug_pec_table  tab: ntab entries of 8 floats (ce x, y, z, pad, ch x, y, z, pad), caller-owned.
 *                         out: 8 (1 + 8 ntab) floats (caller-owned) receive the coded table.  Entry 0
 *                         has ce = 0 and material 0's ch.  Entry 1 + m + ntab f has material m's
 *                         coefficients, with ce set to 0 for each E component tangential to a face in f
 *                         (x to the j = 0 and k = 0 faces, y to i = 0 and k = 0, z to i = 0 and j = 0).
 * Both return FDTD_ERR_ARG for NULL pointers or arguments outside those ranges. */
FDTD_API int fdtd_debug_pec_code(int ntab, int id, int i, int j, int k, int *code);
FDTD_API int fdtd_debug_pec_table(const float *tab, int ntab, float *out);

/*
 * fdtd_energy_static - the same energy W as fdtd_energy (second-order scheme), computed from
 * caller-owned device arrays by a path that allocates no device memory.  (The paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc
 * where they need the energy, e.g. inside work they capture into a CUDA graph,
 * under a fixed pre-reserved memory budget, or in a loop that cannot afford
 * cudaMalloc's implicit synchronisation.)
 *   nx, ny, nz, dt, dx  cavity size and steps as for fdtd_create; nz <= 8191.
 *   f[6]                device pointers to canonical FP32 Ex..Hz (taken as given:
 *                       tangential E is not zeroed here).
 *   ce[3], ch[3]        device pointers to canonical FP32 coefficients, or NULL
 *                       for vacuum (dt/dx).
 *   W                   device pointer to one double that receives the energy.
 *   cuda_stream         stream to run on (NULL = legacy default stream).
 * Asynchronous: W is valid once the stream reaches this point.  Partial sums
 * live in a fixed 64 KiB device array inside the library (one double per z
 * plane), shared by every call: calls whose kernels overlap on the GPU race and
 * must be serialised by the caller.  The first call on a device looks up that
 * array's address (cudaGetSymbolAddress) and should come before any stream
 * capture; the address is looked up again when the device's current CUDA
 * context is no longer the one it was found in (after a cudaDeviceReset).
 * Returns FDTD_ERR_ARG (message via fdtd_last_error(NULL)) for NULL pointers,
 * non-positive sizes, nz > 8191 or a z-plane of more than 2^31 points.
 */
FDTD_API int fdtd_energy_static(int nx, int ny, int nz, double dt, double dx, const float *const f[6],
                                const float *const ce[3], const float *const ch[3], double *W,
                                void *cuda_stream);

/* fdtd_version - library version string. */
FDTD_API const char *fdtd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FDTD_H */
