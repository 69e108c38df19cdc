/*
 * lbm.h - C ABI of liblbm.so: GB300 (sm_103a) time stepping of the two lattice-Boltzmann Maxwell
 * schemes compared in arXiv 2309.08068, the Mendoza-Munoz model (MM, Section II) and the modified
 * Hauser-Verhey model (HV, Section III with the source term of eq. SourceTermHV).
 *
 * One context holds one periodic nx x ny x nz lattice on the current CUDA device. Cells are indexed
 * x + nx * (y + ny * z) (x fastest). Vector fields are component-major: component c of cell i is at
 * [c * n + i]. All device work runs on the context's CUDA stream, in order.
 *
 * Error behaviour: every call returns LBM_OK (0) or a negative LBM_E* code; nothing aborts or
 * traps. lbm_last_error() gives a message for the last failing call on a context. A context is not
 * thread-safe: one host thread at a time.
 *
 * Ownership: the library copies every input array at the call (media, sources, initial fields) and
 * never keeps a caller pointer. Outputs go to caller buffers. Device buffers passed with
 * on_device = 1 must be device (or managed) memory of the context's device.
 */
#ifndef LBM_H
#define LBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

/* Models. LBM_MM: D3Q13 velocities with electric and magnetic distributions, 48 moving + 2 rest
 * populations per cell (Section II). LBM_HV: D3Q7 velocities with a vector electric e_i and a vector
 * magnetic h_i distribution per direction, 36 scalars per cell (Section III). */
enum { LBM_MM = 0, LBM_HV = 1 };

enum {
    LBM_OK = 0,
    LBM_EINVAL = -1,       /* bad argument (null pointer, size, index, unknown enum) */
    LBM_ENOMEM = -2,       /* device or host allocation failed */
    LBM_ECUDA = -3,        /* a CUDA runtime call or kernel launch failed */
    LBM_ENONFINITE = -4,   /* lbm_check_finite found a NaN or infinity */
    LBM_ETIMEDOUT = -5,    /* a bounded wait ran out (a two-step pass's dependency wait) */
    LBM_EUNSUPPORTED = -6  /* valid request this build does not implement */
};

/* Population storage precision; arithmetic is FP32 in every case. LBM_BF16 and LBM_F16 store each
 * population in 16 bits (half the bytes of a bandwidth-bound step) as f * storage_scale, rounded to
 * nearest. Measured on GB300 against the FP64 oracle after the 1500-step dielectric pulse: relative L2
 * error 2-3 % (FP16, scale 2^20) and 10-21 % (BF16); neither keeps FP32's grid-convergence order.
 * LBM_F24 stores 24 bits per population (three quarters of FP32's bytes): f * storage_scale cut
 * toward zero to FP16, plus a byte holding the remainder in 256ths of that half's last place,
 * rounded to nearest (a full 256 moves the half one value on): 19 significant bits, relative error
 * at most 2^-19. Its range is FP16's, so storage_scale must keep |f| * storage_scale below 65504
 * (larger values saturate) and well above 2^-24 for the precision to hold. Measured the same way:
 * 1.2e-4 after the pulse, and FP32's first-order grid convergence kept up to Lz = 4096. No two-step
 * pass and no z_ghost slab takes it (lbm_step runs single steps; lbm_create refuses a z_ghost slab
 * with LBM_EUNSUPPORTED); batches, fields, reductions and population access do. */
enum { LBM_F32 = 0, LBM_BF16 = 1, LBM_F16 = 2, LBM_F24 = 3 };

/* Per-cell linear media (Section I-B remark: eps = eps_r eps0, mu = mu_r mu0). Each pointer is an
 * array of n floats, or NULL for the uniform default eps_r = 1, mu_r = 1, sigma = 0. on_device
 * selects device or host memory for all three. Requirements: eps_r > 0, mu_r > 0, sigma >= 0,
 * finite. When the lattice holds at most 256 distinct (eps_r, mu_r, sigma) triples the library
 * stores one byte per cell and a material table; otherwise it stores the three per-cell arrays. */
typedef struct {
    const float* eps_r;
    const float* mu_r;
    const float* sigma;
    int on_device;
} lbm_media;

/* Context options; pass NULL for all defaults.
 * storage: LBM_F32, LBM_BF16, LBM_F16 or LBM_F24.  cuda_stream: a cudaStream_t, or NULL for the
 *   legacy default stream.
 * storage_scale: 16- and 24-bit storage keep f * storage_scale; a power of two (so scaling is
 *   exact), 0 for 1. FP16 and F24 need it to keep small populations out of subnormals (FP16's
 *   smallest normal is 6.1e-5) and large ones below 65504; BF16 has FP32's range. Ignored for
 *   LBM_F32.
 * track_rho: MM only; also store the rest populations f_0^(0), f_0^(1), so that rho_c (eq.
 *   MacroscopicFieldsMiller) is kept and lbm_get_populations returns them. Otherwise the rest
 *   populations are not stored (neither enters E, B, D, H or J) and read back as 0.
 * eps0, mu0: vacuum constants; 0 selects the model default. MM fixes eps0 = 1, mu0 = 2 (Section
 *   II-A; any other value gives LBM_EUNSUPPORTED). HV default eps0 = mu0 = 3: the paper fixes only
 *   the vacuum speed 1/sqrt(eps0 mu0) = 1/3 (Section III-A), which the split does not change.
 * z_ghost: 1 makes the context one z-slab of a larger lattice (nz >= 3). Planes z = 0 and z = nz - 1
 *   are ghost planes holding the neighbouring slabs' populations: lbm_step updates only the planes
 *   1 .. nz - 2, lbm_reduce and lbm_check_finite sum only those, and sources may not lie in a ghost
 *   plane. Before every step the ghost planes must receive the neighbours' halo (lbm_halo_unpack
 *   or lbm_halo_exchange). A cell's populations are read from its neighbours (pull scheme), so
 *   lbm_fields, lbm_get_populations and lbm_reduce of the boundary planes also need a current halo:
 *   exchange after the last step before reading. The other values of the ghost planes are
 *   unspecified. Not accepted by lbm_batch_create or lbm_adjoint. */
typedef struct {
    int storage;
    void* cuda_stream;
    int track_rho;
    double eps0;
    double mu0;
    double storage_scale;
    int z_ghost;
} lbm_options;

/* Time dependence s(t) of a source, evaluated on the host in double precision for iteration t.
 *   LBM_FN_SIN:   amplitude * sin(2 pi t / period + phase)
 *   LBM_FN_TABLE: amplitude * table[t] for 0 <= t < table_len, else 0 (table copied at the call)
 *   LBM_FN_CONST: amplitude */
enum { LBM_FN_SIN = 0, LBM_FN_TABLE = 1, LBM_FN_CONST = 2 };
typedef struct {
    int kind;
    double amplitude;
    double period;
    double phase;
    const double* table;
    int64_t table_len;
} lbm_time_fn;

/* Sources (Section IV-B/C and the Appendix B note).
 *   LBM_SRC_CURRENT: external current J_ext(x, t) = w(x) s(t) at the listed cells; w holds 3 floats
 *     per cell. MM feeds it to eq. MacroscopicEMiller and the equilibria; HV to J = sigma E + J_ext
 *     and the source term T_i = -(J . v_i) v_i / 2.
 *   LBM_SRC_IMPOSE: after each collision the listed cells are set to the equilibrium of
 *     E = E0 s(t), B = B0 s(t), J = 0 (Appendix B "impose fields"); MM's rest populations keep their
 *     collided values.
 * Several sources may share cells: currents add, imposed fields add. cells[] are in [0, n); host
 * memory; copied at the call. At most LBM_MAX_SOURCES sources per context. */
enum { LBM_SRC_CURRENT = 0, LBM_SRC_IMPOSE = 1 };
#define LBM_MAX_SOURCES 16
typedef struct {
    int kind;
    int64_t n_cells;
    const int64_t* cells;
    const float* w;
    float E0[3];
    float B0[3];
    lbm_time_fn fn;
} lbm_source;

/* Field selection for lbm_fields; output blocks follow in this order, each 3 x n floats. */
enum { LBM_FIELD_E = 1, LBM_FIELD_B = 2, LBM_FIELD_D = 4, LBM_FIELD_H = 8, LBM_FIELD_J = 16 };

/* Create a context for `model` on an nx x ny x nz periodic lattice (every axis >= 1; dimensions of 1
 * are allowed and make that axis trivially periodic). Allocates two population buffers (pull
 * scheme, A/B) on the current device and leaves them zero; t = 0. */
int lbm_create(int model, int nx, int ny, int nz, const lbm_media* media, const lbm_options* opts,
               lbm_ctx** out);

/* Appendix B, first lines: every population := its equilibrium for the given E and B with J = 0
 * (MM: D' = eps_r E, eq. MacroscopicEMiller with J = 0; HV: D = eps0 eps_r E); rest populations 0;
 * t := 0. E and B are 3 x n floats, host (on_device = 0) or device memory. Synchronous for host
 * input; stream-ordered for device input. Host input passes through a device staging buffer that
 * the context keeps for later host-side lbm_init_fields and lbm_fields calls (grown as needed,
 * freed by lbm_destroy); pinned host memory makes the copy fastest. */
int lbm_init_fields(lbm_ctx* ctx, const float* E, const float* B, int on_device);

/* Add one source (see lbm_source). Takes effect from the next lbm_step. */
int lbm_set_source(lbm_ctx* ctx, const lbm_source* src);
/* Remove every source. */
int lbm_clear_sources(lbm_ctx* ctx);

/* Enqueue n >= 0 time steps on the context stream and return without waiting. Iteration t (t = 1,
 * 2, ... counted from lbm_init_fields) evaluates the sources at s(t). Each step is the fused MM or HV
 * update of every cell: pull the neighbours' post-collision populations, form the moments (eqs.
 * MacroscopicFieldsMiller / MacroscopicFieldsHV), compute E and J (eqs. MacroscopicEMiller,
 * MacorscopicCurrentMiller / E = D/eps, J = sigma E + J_ext), the equilibria (eqs.
 * equilibriumsMiller / equilibriumHV), the tau = 1/2 collision (eqs. CollisionMiller /
 * CollisionmodifiedHV), the imposed cells, and store. */
int lbm_step(lbm_ctx* ctx, int n);

/* Fields at the current time t: moments of the current populations, with the external current of
 * iteration t + 1 (the one the next collision uses). For each bit of mask in the order E, B, D, H, J,
 * 3 x n floats are written to out. MM: D = eps0 eps_r E, H = B / (mu0 mu_r). HV: D and B are the
 * moments, E = D / eps, H = B / mu. Host output (on_device = 0) goes through the context's staging
 * buffer (see lbm_init_fields) and waits for the stream; device output is stream-ordered. */
int lbm_fields(lbm_ctx* ctx, unsigned mask, float* out, int on_device);

/* Number of populations per cell in the canonical layout: MM 50, HV 36. */
int lbm_num_populations(int model);

/* Populations f(x, t) before the next collision, canonical layout out[k * n + cell]:
 *   MM: k = r*24 + p*8 + (i-1)*2 + j for the moving ones (r = 0 electric, 1 magnetic; plane p = 0..2;
 *       i = 1..4; j = 0..1, eq. VelocitySetMiller / ElectromagneticVectorsMiller), k = 48: f_0^(0),
 *       k = 49: f_0^(1) (0 unless track_rho).
 *   HV: k = r*18 + (i-1)*3 + c (r = 0: e_i, 1: h_i; i = 1..6 in the Section III order; c = x, y, z).
 * Host output waits for the stream. */
int lbm_get_populations(lbm_ctx* ctx, float* out, int on_device);
/* Load populations in the same layout and set the time to t (checkpoint restore). */
int lbm_set_populations(lbm_ctx* ctx, const float* in, int on_device, int64_t t);

/* Double-precision reductions over the lattice (waits for the stream):
 *   out[0] = field energy (1/2) sum_x (E . D + B . H),  out[1] = sum of squared populations,
 *   out[2] = MM total charge sum_x rho_c (0 unless track_rho; 0 for HV). */
int lbm_reduce(lbm_ctx* ctx, double out[3]);
/* LBM_OK if every stored population is finite, LBM_ENONFINITE otherwise. Waits for the stream. */
int lbm_check_finite(lbm_ctx* ctx);

/* lbm_reduce_noalloc: the same three values as lbm_reduce, computed without allocating any device
 * memory. The paper has no counterpart; this entry point exists for callers that cannot allocate:
 * those whose device memory belongs to a pool of their own, and those whose loop cannot take the
 * implicit synchronisation of cudaMalloc/cudaFree. lbm_reduce may allocate its partial-sum buffer
 * on first use; this call keeps the partial sums in a static device array that every GPU loading the
 * library holds until exit (4096 slots of 3 doubles, 96 KiB). It calls no cudaMalloc or cudaFree.
 *   out: 3 doubles. on_device = 1: device memory, written in stream order (no wait).
 *        on_device = 0: host memory; the call waits for the stream.
 * Limit: the lattice's reduction blocks (at most 608), plus for MM one block per 256 source cells
 *   (about 890,000 source cells on a large lattice), must fit in the 4096 slots; otherwise
 *   LBM_EINVAL with a message giving the limit. HV has no per-source-cell slots.
 * With host output the call first reports, like lbm_reduce, a two-step pass whose dependency wait
 *   ran out (LBM_ETIMEDOUT).
 * The first call on a device looks up the static array's device address (cudaGetSymbolAddress);
 *   make that first call before any stream capture. The address is kept for the life of the
 *   process: after cudaDeviceReset (or anything else that unloads the library's module from the
 *   device) later calls on that device are invalid. Every call, from any context, shares the one
 *   array: nothing in it needs to start at zero, but calls whose kernels overlap on the GPU (for
 *   instance two contexts on different streams) race on it, so order them on one stream or wait in
 *   between. */
int lbm_reduce_noalloc(lbm_ctx* ctx, double* out, int on_device);

/* Number of completed steps. */
int64_t lbm_time(const lbm_ctx* ctx);
/* Kernel launches enqueued by this context so far (all kinds). */
int64_t lbm_launch_count(const lbm_ctx* ctx);
/* Message of the last failing call on ctx (or of the last failing lbm_create when ctx is NULL). */
const char* lbm_last_error(const lbm_ctx* ctx);
/* Wait for the context stream. */
int lbm_sync(lbm_ctx* ctx);
/* Free the context and its device memory. NULL is accepted. */
int lbm_destroy(lbm_ctx* ctx);

/* Two time steps per pass. A step reads only a cell's 3 x 3 x 3 neighbourhood (advection, Sections
 * II and III), so lbm_step(ctx, n >= 2) can run steps t and t + 1 in one launch, reading and writing
 * the populations in HBM once per pair of steps instead of twice. Two such passes exist, and both
 * equal single steps bit for bit (same arithmetic; the intermediate step is held in the context's
 * storage format):
 *   the tiled pass: each block steps a 14 x 14 tile of a chunk of planes plus a ring of one cell
 *   around it (16 x 16 cells, one thread each) twice, keeping the intermediate step in shared
 *   memory as it marches along z; blocks never wait for one another. Needs nx, ny >= 16, nz >= 3.
 *   the ring pass: one persistent launch runs the two steps as a wavefront along z, updating plane
 *   p at step t into a ring of intermediate planes meant to stay in L2, and plane p at step t + 1
 *   once planes p - 1, p, p + 1 of step t exist. Needs a plane of at least 256 cells per SM and
 *   nz >= 4 (MM) or 5 (HV).
 *   mode 0: never; 1 (default): with FP32 storage, the pass measured fastest on GB300: the tiled
 *   pass where its blocks at 8-plane chunks exceed 1.5 waves of resident blocks (smaller lattices
 *   step faster singly), except that HV with a uniform medium takes the ring pass first; else the
 *   ring pass when its intermediate planes (R + 2 planes: R = 5 for MM, 6 for HV) fit in three
 *   quarters of L2; else single steps. 2: the ring pass wherever it applies; 3: the tiled pass
 *   wherever it applies (any storage).
 * Never for z_ghost slabs or track_rho contexts. The ring pass's dependency waits are
 * bounded (2 s, lbm_set_wait_limit); if one expires every block of the pass stops, the populations
 * of that pass are undefined, and the next lbm_sync, lbm_reduce, lbm_reduce_noalloc or host-side
 * lbm_fields / lbm_get_populations returns LBM_ETIMEDOUT (once; until then later passes stop
 * too). After that, restoring populations with lbm_set_populations makes the context usable
 * again. Odd n ends with one single step. The pass
 * allocates its intermediate planes and counters on first use (kept until lbm_destroy).
 * tile_cells: cells per work item of a pass, a multiple of 256 up to 4096; 0 keeps the current
 * value (default 256 for MM, 512 for HV, the fastest on GB300). */
int lbm_set_step_fusion(lbm_ctx* ctx, int mode, int tile_cells);
/* Limit of each dependency wait of a two-step pass, in nanoseconds: ns > 0 sets it, ns == 0 restores
 * the default of 2 s. ns < 0 makes every item of a pass that depends on another give up at its
 * first check, whether its inputs are there or not, so that a test can drive the time-out path
 * deterministically: the pass stops and the next waiting call returns LBM_ETIMEDOUT. Takes effect
 * from the next pass. */
int lbm_set_wait_limit(lbm_ctx* ctx, long long ns);
/* How lbm_step would run pairs of steps: 0 as single steps, 1 as ring passes, 2 as tiled passes
 * (negative on error). */
int lbm_step_fusion_active(lbm_ctx* ctx);
/* Self-check of the two-step pass's work order on the host, with the kernel's own order and tile
 * window functions, for an nx x ny x nz lattice, ring R, lookahead L and tile_cells per item
 * (nx * ny <= 2^22). Checks:
 *   1. every phase appears once;
 *   2. each phase's waits target earlier phases;
 *   3. a ring slot is rewritten only after the readers of its previous plane;
 *   4. a tile's window holds every cell its cells pull from, and windows are symmetric.
 * Returns 0 when all hold, the number of the first failed check otherwise, LBM_EINVAL for bad
 * sizes. Needs no GPU. */
int lbm_fused_schedule_check(int nx, int ny, int nz, int R, int L, int tile_cells);
/* Self-check of the tiled pass's geometry on the host, with the kernel's own tile functions, for an
 * nx x ny plane (nx, ny >= 16, nx * ny <= 2^22). Checks:
 *   1. the 16 x 16 positions of an extended tile are distinct cells;
 *   2. the 3 x 3 neighbours of a tile's own cell lie in its extended tile and are the cell's lattice
 *      neighbours (periodic);
 *   3. the tiles' own cells cover the plane exactly once.
 * Returns 0 when all hold, the number of the first failed check otherwise, LBM_EINVAL for bad
 * sizes. Needs no GPU. */
int lbm_tiled_layout_check(int nx, int ny);

/* Loss and gradient over the next `steps` time steps (inverse material design; the paper itself
 * only runs forward). From the current populations, the context advances `steps` steps exactly as
 * lbm_step does, and
 *   L = sum_{t=1..steps} sum over the cells of plane (plane_axis, plane_index) of |E(t)|^2,
 * with E(t) the field lbm_fields reports after t steps. The gradients dL/d eps_r and dL/d sigma of
 * every cell (n floats each; NULL skips one, and a NULL grad_sigma also skips summing it) are taken
 * at fixed starting populations. The adjoint
 * steps back through the transposed collide-and-stream map. What it needs of forward step t is a
 * per-cell record: X = D' - mu0 J_ext / 4 for MM (E follows from X and the medium), E for HV (12
 * bytes per cell each).
 * The steps are cut into segments of K = checkpoint_interval steps, counted from the end (the first
 * segment may be shorter). The forward pass writes the records of the final segment and keeps the
 * population state at the start of every earlier one; going backward, each earlier segment is
 * recomputed once from its state, writing its records, before it is stepped back through. Work
 * space: K records + one state per earlier segment + 4 states.
 *   checkpoint_interval < 0 (or >= steps): K = steps, every record resident, nothing recomputed.
 *   checkpoint_interval > 0: that K.
 *   checkpoint_interval == 0: resident when its work space fits in half the free device memory,
 *     else K = lbm_adjoint_sqrt_interval(ctx, steps).
 * Every mode gives the same loss and gradients, bit for bit. Needs FP32 storage; source cells must
 * not lie in the plane (LBM_EINVAL). loss_out is a host double; gradient outputs are host
 * (on_device = 0) or device memory. The work space (records or checkpoints, two adjoint states, the
 * gradient sums) is allocated on the first call, LBM_ENOMEM when it does not fit, and kept by the
 * context for later calls, which grow it when they need more; lbm_adjoint_release or lbm_destroy
 * frees it. Waits for the stream. */
int lbm_adjoint(lbm_ctx* ctx, int steps, int plane_axis, int plane_index, int checkpoint_interval, double* loss_out,
                float* grad_eps_r, float* grad_sigma, int on_device);
/* Free the work space lbm_adjoint keeps (after waiting for the stream). */
int lbm_adjoint_release(lbm_ctx* ctx);
/* Bytes of device memory held as lbm_adjoint work space (0 when none; -1 for NULL). */
int64_t lbm_adjoint_workspace_bytes(const lbm_ctx* ctx);
/* Segment length of the checkpointed mode for `steps` steps: the longest K whose work space stays
 * within that of segments of ceil(sqrt(steps)) steps (about sqrt(steps) states and as many
 * records, the classic sqrt(T) layout), so the memory grows like sqrt(steps). A record (12 B per
 * cell) is 16 (MM) or 12 (HV) times smaller than a state, so this K is several times sqrt(steps),
 * and the forward pass records that many final steps instead of recomputing them. LBM_EINVAL
 * (negative) for bad arguments. */
int lbm_adjoint_sqrt_interval(const lbm_ctx* ctx, int steps);

/* ---------------------------------------------------------------------------------------------
 * z-slab decomposition. The scheme couples a cell only to its 3 x 3 x 3 neighbourhood (Sections II
 * and III, advection), so a lattice can be split into slabs along z that exchange one plane of
 * populations per face and step. A slab context (z_ghost = 1) has one ghost plane at each end. After
 * a step, the values that leave a slab through a face are the post-collision populations of its
 * boundary plane in the directions that cross that face. The pull scheme stores them at the cell
 * that produced them, so they are copied unchanged into the neighbour's ghost plane:
 *   face 1 (up): plane nz - 2, directions with v_z = +1 (MM groups 4, 5, 8, 9; HV direction +z),
 *     which the upper neighbour reads from its plane 0;
 *   face 0 (down): plane 1, directions with v_z = -1 (MM groups 6, 7, 10, 11; HV direction -z),
 *     which the lower neighbour reads from its plane nz - 1.
 * A packed face is those directions' planes one after another, each nx * ny cells in the context's
 * storage layout: MM 4 x 16 B per cell in FP32 (8 B in 16-bit storage); HV 16 B + 8 B (8 B + 4 B).
 * MM's rest populations do not move and are not exchanged. Slabs stepped this way give the same
 * populations, bit for bit, as the unsplit lattice.
 * ------------------------------------------------------------------------------------------- */
/* Bytes of one packed face (z_ghost contexts; LBM_EINVAL otherwise, as a negative value). */
int64_t lbm_halo_bytes(const lbm_ctx* ctx);
/* Pack the outgoing values of face 0 or 1 of the current state into dst (lbm_halo_bytes bytes;
 * device memory when on_device, else host memory and the call waits for the stream). */
int lbm_halo_pack(lbm_ctx* ctx, int face, void* dst, int on_device);
/* Write a face packed by the neighbour into ghost plane 0 (face 0: the lower neighbour's face 1) or
 * nz - 1 (face 1: the upper neighbour's face 0) of the current state. */
int lbm_halo_unpack(lbm_ctx* ctx, int face, const void* src, int on_device);
/* Both directions across the interface between `lower` (whose face 1 it is) and `upper` (face 0),
 * on one device, in one kernel: lower's face 1 into upper's plane 0, upper's face 0 into lower's
 * plane nz - 1. The contexts must have the same model, storage, nx, ny, device and stream;
 * lower == upper closes a single slab periodically. Stream-ordered. */
int lbm_halo_exchange(lbm_ctx* lower, lbm_ctx* upper);

/* ---------------------------------------------------------------------------------------------
 * Batched stepping of lattices of uneven sizes. The paper's studies are mesh-refinement sweeps:
 * the same test on lattices refined step by step (Section IV, "for different refinements of the
 * grid"). A batch advances all of them together, one fused launch per time step over every active
 * lattice, and replays the whole sequence as one captured CUDA graph. A small lattice alone cannot
 * fill the GPU, so batching is what keeps it busy.
 * ------------------------------------------------------------------------------------------- */
typedef struct lbm_batch lbm_batch;

/* Group count >= 1 distinct contexts of the same model, storage, track_rho, CUDA stream and device.
 * The batch keeps the pointers: the contexts stay owned by the caller and must outlive the batch.
 * Sources and populations may still be changed between calls through the context API. */
int lbm_batch_create(lbm_ctx* const* ctxs, int count, lbm_batch** out);

/* Advance context k by steps[k] >= 0 time steps (results identical, bit for bit, to lbm_step on each
 * context). A context for which lbm_step would run two steps per pass (lbm_set_step_fusion) runs its
 * steps exactly that way, through direct launches. Step j of the call updates every other context
 * with steps[k] > j in one launch (plus one launch for source cells); each context's time and
 * sources advance as in lbm_step. On a non-default stream the
 * whole call is captured once into a CUDA graph and replayed by later calls with the same steps,
 * sizes and source-cell counts; on the legacy default stream the launches are issued directly.
 * Asynchronous: enqueued on the contexts' stream. */
int lbm_batch_step(lbm_batch* b, const int* steps);

/* Time trial_steps launches of each launch configuration (128 or 256 threads per block; one block
 * per tile, or a persistent grid of resident blocks striding over the tiles) on this batch and keep
 * the fastest. The trial launches rewrite only the spare population buffers, so the lattices' state
 * is unchanged. Waits for the stream. The chosen configuration is returned when the pointers are
 * non-NULL. */
int lbm_batch_autotune(lbm_batch* b, int trial_steps, int* block_out, int* persistent_out);

/* Set the launch configuration directly: block is 128 or 256, persistent 0 or 1. */
int lbm_batch_set_config(lbm_batch* b, int block, int persistent);

/* Kernel launches enqueued by the batch so far (graph replays count their kernels). */
int64_t lbm_batch_launch_count(const lbm_batch* b);
/* Message of the last failing batch call (or of the last failing lbm_batch_create when b is NULL). */
const char* lbm_batch_last_error(const lbm_batch* b);
/* Free the batch (not its contexts). NULL is accepted. */
int lbm_batch_destroy(lbm_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
