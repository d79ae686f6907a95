/*
 * pme.h — C ABI of the GB300 reciprocal-space Smooth Particle Mesh Ewald (SPME) library.
 *
 * The library evaluates the long-range (reciprocal-space) part of Ewald electrostatics by SPME, the
 * pipeline the paper runs on its FPGA cluster (Sec. III-A, "Long-Range Pipeline"): B-spline charge
 * spreading onto a K1 x K2 x K3 mesh (Sec. III-A "Charge Spreading"), a forward 3D FFT, a multiply by the
 * influence ("Green's") function, an inverse 3D FFT (Sec. III-A "FFT"), and force interpolation with the
 * B-spline derivatives (Sec. III-A "Force Interpolation"). Energy and virial are reduced on the fly in
 * the influence-function step. The equations are the standard SPME ones [Essmann et al. 1995], which
 * the paper cites for the method (Sec. II) without writing them out:
 *   E = 1/2 sum_{m != 0} B(m) C(m) |FFT(Q)(m)|^2,
 *   C(m) = exp(-pi^2 |m'|^2 / beta^2) / (pi V |m'|^2),  B(m) = prod_alpha |b_alpha(m_alpha)|^2,
 *   Pi_ab = 1/2 sum B C |FFT(Q)|^2 (delta_ab - 2 (1 + pi^2 |m'|^2 / beta^2) m'_a m'_b / |m'|^2),
 *   F_i = -q_i sum_k grad_i[theta_1 theta_2 theta_3](k) phi(k),  phi = IFFT(B C FFT(Q)).
 *
 * Only the reciprocal-space term is computed: the caller adds the real-space and self terms.
 *
 * Units: lengths in Angstrom, charges in e, Coulomb constant 1: energy and virial in e^2/A, forces in
 * e^2/A^2. Multiply by 332.0637 for kcal/mol.
 *
 * Conventions for every call:
 *   - Array arguments are DEVICE pointers on the plan's device (for example a torch CUDA tensor's
 *     data_ptr()), unless the function name ends in _host. Scalars returned through pointers
 *     (energy, virial) are host pointers unless stated otherwise.
 *   - pos is n x 3 float32, row-major (x, y, z per atom); any position is accepted and wrapped into
 *     the periodic cell. q is n float32. forces is n x 3 float32, overwritten.
 *   - virial[6] = (xx, yy, zz, xy, xz, yz).
 *   - The caller owns all input/output arrays; the library owns plans, meshes, tables and scratch.
 *   - No call aborts, throws across the ABI or traps on the device. Errors come back as pme_status;
 *     pme_last_error_detail() gives a message for the last error on the calling thread.
 *   - A plan is not thread-safe: one host thread (or external locking) per plan.
 */
#ifndef PME_GB300_H
#define PME_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pme_plan pme_plan;      /* opaque: one periodic system geometry + its resident device state */
typedef struct pme_batch pme_batch;    /* opaque: a fixed set of systems evaluated together per call */
typedef struct pme_server pme_server;  /* opaque: continuous-batching request loop */
typedef int64_t pme_ticket;

typedef enum {
    PME_OK = 0,
    PME_EINVAL = 1,        /* invalid argument, or a non-finite / absurdly far position or charge */
    PME_EUNSUPPORTED = 2,  /* valid SPME parameters this build does not implement (e.g. p = 7) */
    PME_ENOMEM = 3,        /* device or host allocation failed, or over the server memory budget */
    PME_ECUDA = 4,         /* a CUDA runtime call failed (detail has the CUDA error string) */
    PME_EOVERFLOW = 5,     /* sum |q| too large for the 64-bit fixed-point charge mesh */
    PME_EAGAIN = 6,        /* server: no slot or memory free right now; retry later */
    PME_ETIMEOUT = 7,      /* a bounded device-side wait gave up (persistent work-list kernel dependency) */
    PME_PENDING = 8        /* pme_poll: request still in flight */
} pme_status;

/* ------------------------------------------------------------------------------------------------------ */
/* Single system                                                                                           */

/* Paper: Sec. III-A (Long-Range Pipeline) and its "Charge Spreading" and "FFT" parts fix what a plan holds:
 * the mesh of K1 x K2 x K3 points the charges are spread onto with order-p cardinal B-splines, and the
 * Green's-function (influence) data multiplied between the forward and inverse transforms, which the paper
 * keeps resident in HBM (Sec. V-C). */
/* Create a plan for mesh K[3] (K1, K2, K3), B-spline order p, Ewald splitting parameter beta (1/A) and
 * periodic cell box[9] (rows are the cell vectors a, b, c in A; any non-singular, right- or left-handed
 * cell). cuda_stream is a cudaStream_t (NULL = the legacy default stream) on the current device; every
 * launch of the plan goes to it.
 * Requirements: each K_alpha even, 8 <= K_alpha <= 128 and with no prime factor other than 2, 3, 5;
 * p in {4, 5, 6, 8} and p <= min(K); beta > 0 and finite. Invalid values return PME_EINVAL; other orders
 * return PME_EUNSUPPORTED. For the odd order the B-spline modulus denominator, which vanishes at m = K/2,
 * takes the mean of its two neighbours there. The plan precomputes the influence-function table B(m)C(m) in FP64 (stored as an
 * unevaluated sum of two floats) and the FFT twiddles, and allocates the mesh (about 30 bytes per mesh
 * point). On success *out receives the plan; on failure *out is NULL. */
pme_status pme_create(const int K[3], int p, double beta, const double box[9], void *cuda_stream, pme_plan **out);

/* Paper: Sec. III-A "FFT" (the Green's-function data multiplied between the transforms depends on the cell
 * through |m'| and V) and Sec. V-C (that data is kept in device memory, so a new cell rewrites it). */
/* Replace the periodic cell (e.g. after a barostat step); recomputes the influence table. Same box
 * rules as pme_create. Synchronous with respect to the plan stream. */
pme_status pme_set_box(pme_plan *plan, const double box[9]);

/* Paper: Sec. III-A (Long-Range Pipeline): each timestep takes atom positions and charges and returns the
 * long-range force on every atom, through charge spreading, the forward 3D FFT, the Green's-function
 * multiply, the inverse 3D FFT and force interpolation with the B-spline derivatives. Energy and virial
 * are the standard SPME sums over the same spectrum (the method the paper cites in Sec. II). */
/* One SPME evaluation, synchronous: enqueues the pipeline on the plan stream, waits for it, and returns
 * energy (host double*) and virial (host double[6]); either may be NULL. n = 0 gives energy 0, virial 0.
 * A call with the same arrays and n as the previous one records the six stages and the kernel that writes
 * energy, virial and status to host memory as one CUDA graph, which later identical calls replay.
 * pos, q, forces are device pointers (see conventions). The first call with a given n (or a larger n
 * than before) may allocate per-atom scratch; later calls allocate nothing. Returns PME_EINVAL for a
 * non-finite position or charge, PME_EOVERFLOW when sum |q| >= 2^22 e (the fixed-point mesh headroom);
 * in both cases the outputs are unspecified. */
pme_status pme_compute(pme_plan *plan, const float *pos, const float *q, int64_t n, float *forces, double *energy,
                       double *virial);

/* Paper: Sec. III-A "Charge Spreading" (the FFT input volume it builds) and "FFT" (the potential mesh the
 * inverse transform hands to force interpolation). */
/* pme_compute with diagnostic taps: when non-NULL, mesh_dev (DEVICE, K1*K2*K3 int64, [k1][k2][k3] with k3
 * fastest) receives the charge mesh after spreading as fixed-point integers round(Q * 2^40) summed
 * exactly, and phi_dev (DEVICE, K1*K2*K3 float) the potential mesh phi after the inverse FFT. Meant for
 * verification (stage-by-stage comparison, bit-exactness of the mesh); costs two extra copies. */
pme_status pme_compute_debug(pme_plan *plan, const float *pos, const float *q, int64_t n, float *forces,
                             double *energy, double *virial, int64_t *mesh_dev, float *phi_dev);

/* Paper: Sec. III (System Architecture): many timesteps run on the accelerator with no host traffic beyond
 * initialization and result collection; this call enqueues one timestep's evaluation without a host wait. */
/* Asynchronous form of pme_compute: enqueues the pipeline and returns without waiting. ev_dev is a
 * DEVICE pointer to 7 doubles that receives (energy, virial[6]) when the stream reaches that point.
 * Allocates nothing once pme_reserve(plan, n) (or an earlier call with at least n atoms) has run, so it
 * may be captured in a CUDA graph. Device-side errors are latched in the plan and returned by the next
 * pme_sync(). */
pme_status pme_enqueue(pme_plan *plan, const float *pos, const float *q, int64_t n, float *forces, double *ev_dev);

/* Paper: Sec. III (initialization before the timestep loop, so the loop itself needs no host work). */
/* Pre-allocate per-atom scratch for up to n atoms (so later pme_enqueue calls allocate nothing). */
pme_status pme_reserve(pme_plan *plan, int64_t n);

/* Paper: Sec. III (result collection after the timesteps the accelerator ran on its own). */
/* Wait for the plan stream and return (and clear) any device-side error latched by enqueued work. */
pme_status pme_sync(pme_plan *plan);

/* Paper: Sec. III-A (Long-Range Pipeline) with the host application of Fig. "MDOverview" on the other side:
 * positions and charges come from host memory and the forces go back to it every timestep. */
/* pme_compute with HOST arrays (pos, q, forces in pageable or pinned host memory): the library copies
 * inputs to its own device staging, evaluates, and copies forces back, all on the plan stream, and
 * returns when forces, energy and virial are in host memory. When all three arrays are page-locked
 * (cudaHostAlloc / cudaHostRegister), no copy engine is used: the binning kernel reads positions and charges
 * in host memory over the CPU-GPU link, and one copy kernel writes the forces (from device staging) and the
 * control block to host memory; a call with the same arrays and n as the previous one records the stages
 * and that kernel as one CUDA graph, which later identical calls replay (one launch per call). The arrays
 * must then stay page-locked and allocated while the plan uses them. */
pme_status pme_compute_host(pme_plan *plan, const float *pos, const float *q, int64_t n, float *forces,
                            double *energy, double *virial);

/* Paper: Sec. III (many timesteps without host round trips) with the host application of Fig. "MDOverview":
 * the asynchronous form of pme_compute_host. pos, q, forces (n x 3) and result (8 doubles) must all be
 * page-locked host memory (cudaHostAlloc / cudaHostRegister), else PME_EINVAL. Enqueues the evaluation and
 * returns its ticket in *ticket (may be NULL; tickets count the plan's calls from 0). The plan keeps two
 * device slots (positions, charges, forces), used alternately: on a stream of the plan's own the copy
 * engine brings the inputs into the slot once the evaluation that last used it has finished; the plan
 * stream waits for them and evaluates; then the copy engine takes the forces and result[0..6] = (energy,
 * virial[6]), result[7] = the device status bits (0: no error) out on a second stream of the plan's own. So
 * the copies of one evaluation overlap the evaluation before or after it. The results of ticket t are in host
 * memory once pme_host_wait(plan, t) returns (or pme_sync). A caller keeps evaluations in flight on several
 * sets of arrays and waits for the older ticket before reusing its set. Each slot's evaluation is recorded
 * once as a CUDA graph, whatever host arrays the calls name. All four arrays
 * must stay allocated and unchanged until the ticket has completed. Not callable while the plan stream is
 * being captured into a graph. */
pme_status pme_enqueue_host(pme_plan *plan, const float *pos, const float *q, int64_t n, float *forces,
                            double *result, int64_t *ticket);

/* Blocks until the forces and result of pme_enqueue_host's ticket are in host memory. PME_EINVAL for a
 * ticket the plan has not issued. Device errors are reported through result[7] (and by pme_sync). */
pme_status pme_host_wait(pme_plan *plan, int64_t ticket);

/* Paper: Sec. V-B and V-C, which time the stages of the pipeline separately (Table IV brackets the forward
 * and inverse FFTs with timestamps). */
/* Per-stage device time: runs reps evaluations, each stage kernel bracketed by CUDA events on the plan
 * stream, and returns the mean microseconds per stage in stage_us[6] = (bin, spread, forward FFT,
 * influence multiply + energy/virial, inverse FFT, force interpolation). Arrays as in pme_compute;
 * forces receive the last evaluation's result. Synchronous. */
pme_status pme_profile_stages(pme_plan *plan, const float *pos, const float *q, int64_t n, float *forces, int reps,
                              double stage_us[6]);

/* Paper: Sec. III-A (Fig. "LRPipe"): the stages are pipelined, each starting on its input while the one
 * before it drains; on this GPU that overlap is programmatic dependent launch between the stage kernels. */
/* Launch option of the stage kernels (process-wide, for launches issued afterwards): 0 = plain stream
 * order; 1 = programmatic dependent launch, each kernel letting its successor launch as soon as it starts;
 * 2 (default) = the same, released as each CTA finishes (the influence stage releases the inverse FFT
 * stage right after its own wait, which measured faster); 3 = released right after each CTA's own wait
 * for its predecessor. Every kernel still waits for its predecessor to complete before touching data, so
 * results are identical in all modes; only launch latency overlap differs. Returns PME_EINVAL for other
 * values. */
pme_status pme_set_launch_mode(int mode);

/* Paper: Sec. III-A ("FFT"): each slab of the 3D transform is a 2D transform of one mesh plane; the paper
 * gives each slab a pipeline. Here: how many CTAs (SMs) transform one slab in the forward (fwd_ctas) and
 * in the inverse (inv_ctas) slab stage of single-system evaluations (process-wide, for launches issued
 * afterwards): 1, or 2 / 4 CTAs forming a thread-block cluster that exchanges its intermediate rows or
 * columns through distributed shared memory. Meshes with K2 = K3 in {32, 64, 128} have the 2-CTA kernels,
 * K2 = K3 = 64 the 4-CTA ones; other meshes keep one CTA per slab. The default is 1 and 1: split slabs
 * measured slower in the pipelined evaluation (their stage alone can be faster). Results are bitwise the
 * same for every value. Returns PME_EINVAL for other values. */
pme_status pme_set_slab_split(int fwd_ctas, int inv_ctas);

/* Paper: Sec. V-C (which problem sizes fit in on-chip memory and which need HBM); here the figure the
 * serving loop admits requests by. */
/* Paper: Sec. VI lists reduced precision among the future work. How the influence stage (the k1 transforms
 * around the Green's-function multiply) computes, for single-system evaluations of this plan
 * (pme_compute, pme_enqueue, pme_compute_host, pme_profile_stages, pme_run_steps; batches and the server
 * always use the FP32 stage):
 *   PME_INFLUENCE_FP32   (default) 128-point FFTs in FP32 registers;
 *   PME_INFLUENCE_TENSOR the transforms as dense matrix products on the tensor cores (tcgen05, BF16 inputs,
 *                        FP32 accumulation), every operand split into three BF16 terms (about 24 bits),
 *                        the six term products above 2^-24 kept; K1 = 128 only (else PME_EUNSUPPORTED).
 * Both give the same results within FP32 rounding; the energy, virial and forces stay within the tolerances
 * against the FP64 reference. The first switch to the tensor path uploads a 192 KB matrix image.
 * Synchronous with respect to the plan stream. */
enum { PME_INFLUENCE_FP32 = 0, PME_INFLUENCE_TENSOR = 1 };
pme_status pme_set_influence_path(pme_plan *plan, int path);
/* The plan's influence path, or -1 for a NULL plan. */
int pme_get_influence_path(const pme_plan *plan);

/* Device bytes the plan holds right now (mesh, tables, per-atom scratch). */
size_t pme_plan_device_bytes(const pme_plan *plan);

/* Releases everything pme_create and later calls allocated for the plan. The plan must be idle. */
void pme_destroy(pme_plan *plan);

/* Allocation-free evaluation of one small system, for callers that must not allocate device memory:
 * applications that gave all device memory to their own pool at start-up (nothing may be left for
 * cudaMalloc), and latency-bound callers that cannot afford the device-wide synchronisation cudaMalloc and
 * cudaFree imply. The paper has no counterpart; it is an interface for such callers.
 * The caller passes only inputs and outputs, as in pme_compute (device pos, q, forces; host energy and
 * virial, either may be NULL); K, p, beta and box follow the pme_create rules. Everything else (meshes,
 * spectrum, influence table, recomputed on the device every call, bucket lists, counters) lives in one
 * static device array of 4 MiB that every GPU loading the library holds until the process exits.
 * Limits: K1*K2*K3 <= 32768 with each K_alpha <= 64, n <= 16384, and the carved scratch must fit in 4 MiB;
 * anything larger returns PME_EINVAL with the reason. One cooperative kernel launch on cuda_stream, then the
 * call waits for it. The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * and the cooperative grid size, so make that first call before any stream capture. Every call starts by
 * clearing the parts of the array that must be zero, but all calls share the one array: calls that overlap
 * on the GPU (from different streams or threads) race and give wrong results. */
pme_status pme_compute_noalloc(const int K[3], int p, double beta, const double box[9], const float *pos,
                               const float *q, int64_t n, float *forces, double *energy, double *virial,
                               void *cuda_stream);

/* ------------------------------------------------------------------------------------------------------ */
/* Autotuning of the launch configuration                                                                  */

/* Paper: Sec. IV-A and Table III size the FFT and spreading pipelines to each problem size on the FPGA; the
 * GPU counterpart is choosing, per mesh and atom density, the spreading / force-interpolation tile edge
 * (8^3 or 16^3 mesh points) and CTA size (128 or 256 threads; 256 or 512 with 16^3 tiles). Every such choice
 * gives bit-identical results (an exact integer charge mesh; each atom's force summed over its support in a
 * fixed order), so tuning changes only speed. */
typedef struct {
    int tile_edge;       /* chosen tile edge (8 or 16 mesh points) */
    int tile_threads;    /* chosen spread / force CTA size (0: the default sizes, which differ per stage;
                          * else 128, 256, or 512 with 16^3 tiles, for both stages) */
    double us_per_eval;  /* its time per evaluation (0 when taken from the cache) */
    double default_us;   /* the default configuration's time (0 when taken from the cache) */
    int candidates;      /* configurations tried */
    int rejected;        /* configurations whose results differed from the default's (never expected) */
    int from_cache;      /* 1 when the choice came from the cache file */
} pme_tune_result;
enum { PME_TUNE_FORCE = 1 };

/* Choose the plan's configuration for n atoms like these: unless flags has PME_TUNE_FORCE, a choice cached
 * for (device, mesh, order, atoms-per-tile class) is applied; otherwise every candidate runs reps timed
 * evaluations (CUDA events on the plan stream) on the caller's DEVICE arrays pos, q, forces (forces receive
 * the last result), its results are compared bit for bit with the default configuration's, and the fastest
 * identical one is kept for the plan and written to the cache. Synchronous; do not call while capturing a
 * graph. out (host) may be NULL. */
pme_status pme_autotune(pme_plan *plan, const float *pos, const float *q, int64_t n, float *forces, int reps, int flags,
                        pme_tune_result *out);

/* Cache file of tuned choices (JSON, read on first use and rewritten after each tuning); NULL or "" keeps
 * choices in memory only. Process-wide. */
pme_status pme_tune_cache(const char *path);

/* Set the plan's tile edge (0 = default: 16 where the 16^3 tiling has at least two tiles per SM and about
 * 256 atoms per tile or more, else 8) and spread / force CTA size (0 = the defaults, chosen per stage by
 * tile edge and atom density; else 128 or 256, or 512 with tile edge 16, for both stages) by hand; the
 * current configuration is reported by pme_plan_get_tiling (tile_threads 0: the defaults). Batches built on
 * the plan pick the change up at their next pme_batch_enqueue. */
pme_status pme_plan_set_tiling(pme_plan *plan, int tile_edge, int tile_threads);
pme_status pme_plan_get_tiling(const pme_plan *plan, int *tile_edge, int *tile_threads);

/* ------------------------------------------------------------------------------------------------------ */
/* Real-space and self terms (the rest of the Ewald sum)                                                   */

/* Paper: Sec. II splits the electrostatics by the Ewald method into the long-range part SPME evaluates and
 * a short-range real-space pair sum, which the paper's system computes on its own pipelines beside the
 * long-range one (Sec. III, Fig. "MDOverview"). These calls evaluate that pair sum and the self term on the
 * GPU, so that E = E_rec (pme_compute) + E_real + E_self is the full Ewald energy of point charges:
 *   E_real = 1/2 sum_{i,j,n}' q_i q_j erfc(beta r) / r  over all periodic images with r = |r_i - r_j + n| <= rcut
 *            (the primed sum skips i = j in the home cell),
 *   F_i    = sum' q_i q_j [erfc(beta r) / r + 2 beta / sqrt(pi) exp(-beta^2 r^2)] (r_i - r_j + n) / r^2,
 *   Pi_ab  = 1/2 sum' q_i q_j [erfc(beta r) / r + 2 beta / sqrt(pi) exp(-beta^2 r^2)] d_a d_b / r^2,
 *   E_self = -beta / sqrt(pi) sum_i q_i^2.
 * Units as for pme_compute. Use the same beta as the reciprocal plan. */
typedef struct pme_real pme_real;  /* opaque: cell grid and scratch of one periodic cell */

/* Create a real-space context for cell box[9] (rows a, b, c), splitting parameter beta (1/A) and cutoff
 * rcut (A), launching on cuda_stream (NULL = legacy default stream) of the current device. Any cutoff up to
 * four cell widths along each axis works (images of an atom itself included); a larger one, or a cell grid
 * over 2^22 cells, returns PME_EUNSUPPORTED. Invalid values return PME_EINVAL. */
pme_status pme_real_create(const double box[9], double beta, double rcut, void *cuda_stream, pme_real **out);

/* Replace the cell (same rules as pme_real_create). Synchronous with respect to the context's stream. */
pme_status pme_real_set_box(pme_real *rs, const double box[9]);

/* Pre-allocate per-atom scratch for up to n atoms, so pme_real_enqueue allocates nothing afterwards. */
pme_status pme_real_reserve(pme_real *rs, int64_t n);

/* Asynchronous evaluation on DEVICE arrays pos (n x 3), q (n), forces (n x 3): the real-space forces are
 * written to forces (accumulate = 0) or added to it (accumulate != 0, e.g. after pme_enqueue on the same
 * stream wrote the reciprocal forces). When ev_dev (DEVICE, 8 doubles) is not NULL it receives (E_real,
 * E_self, virial[6]) when the stream reaches that point. Results are bit-reproducible run to run and do not
 * depend on the order of the atoms except through the summation order of each atom's neighbours. */
pme_status pme_real_enqueue(pme_real *rs, const float *pos, const float *q, int64_t n, float *forces, int accumulate,
                            double *ev_dev);

/* Synchronous evaluation: forces (DEVICE, overwritten), and on the host e_real, e_self and virial[6]
 * (either may be NULL). Returns PME_EINVAL for a non-finite or absurdly far position or charge. */
pme_status pme_real_compute(pme_real *rs, const float *pos, const float *q, int64_t n, float *forces,
                            double *e_real, double *e_self, double *virial);

/* Release the context (it must be idle). */
void pme_real_destroy(pme_real *rs);

/* ------------------------------------------------------------------------------------------------------ */
/* One system over several ranks: slab decomposition with two corner turns                                 */

/* Paper: Sec. III-A "FFT", III-C and IV-C: the mesh is divided into slabs, each transformed independently;
 * an all-to-all "corner turn" regroups the data so that every pipeline holds full pencils for the
 * Green's-function multiply, and a second one returns it; atoms that affect several pipelines are processed
 * by each of them (Sec. III-A "Charge Spreading"). Here rank r of nranks owns a contiguous range of mesh
 * planes along k1 and of influence-stage columns (pme_slab_layout); one evaluation is
 *   pme_slab_stage1 -> all-to-all -> pme_slab_stage2 -> all-to-all -> pme_slab_stage3,
 * then the caller sums the ranks' forces and energy / virial partials. The all-to-alls are the caller's
 * (for example torch.distributed.all_to_all_single over NCCL): send and recv are DEVICE buffers of nranks
 * equal blocks of block_values complex FP32 values (2 floats each), block s of send going to rank s and block
 * r of recv coming from rank r. Every call enqueues on the rank's stream and returns without waiting;
 * nothing waits on another rank. Results equal the undivided evaluation within FP32 rounding (the force
 * and energy sums are split across ranks). */
typedef struct pme_slab pme_slab;

/* Rank `rank` of `nranks` for mesh K, order p, beta, cell box (pme_create rules), on cuda_stream. Returns
 * PME_EUNSUPPORTED when the mesh cannot give every rank a plane and an influence item. */
pme_status pme_slab_create(const int K[3], int p, double beta, const double box[9], int nranks, int rank,
                           void *cuda_stream, pme_slab **out);
/* The rank's planes [planes[0], planes[1]) and half-spectrum columns [columns[0], columns[1]) (c = m2 (K3/2 + 1)
 * + m3), and the complex values per exchange block; any pointer may be NULL. */
pme_status pme_slab_layout(const pme_slab *slab, int *planes, int *columns, int64_t *block_values);
/* Stage 1 on DEVICE pos (n x 3) and q (n), all atoms of the system on every rank: binning, spreading into the
 * own planes, forward slab transforms of those planes, and the first exchange's send blocks. */
pme_status pme_slab_stage1(pme_slab *slab, const float *pos, const float *q, int64_t n, float *send);
/* Stage 2: the first exchange's recv blocks in; the influence stage on the own columns; this rank's partial
 * (E, virial[6]) to ev_dev (DEVICE, 7 doubles; NULL keeps it internal); the second exchange's send blocks. */
pme_status pme_slab_stage2(pme_slab *slab, const float *recv, float *send, double *ev_dev);
/* Stage 3: the second exchange's recv blocks in; inverse slab transforms of the own planes; forces (DEVICE,
 * n x 3, overwritten) = the part of every atom's force from the own planes (same pos, q, n as stage 1). */
pme_status pme_slab_stage3(pme_slab *slab, const float *recv, const float *pos, const float *q, int64_t n,
                           float *forces);
/* Wait for the rank's stream and report (and clear) device-side errors. */
pme_status pme_slab_sync(pme_slab *slab);
void pme_slab_destroy(pme_slab *slab);

/* ------------------------------------------------------------------------------------------------------ */
/* Multi-step loop on the device                                                                           */

/* Paper: Sec. III runs multiple timesteps on the accelerators with no host communication beyond
 * initialization and result collection. This call enqueues `steps` time steps on the plan stream, each:
 * reciprocal-space forces of the plan into forces, plus (when rs is not NULL) the real-space forces of rs
 * added to them, then a leapfrog update
 *     v += (F * inv_mass) * dt,   x += v * dt     (each product and sum rounded once in FP32),
 * all on DEVICE arrays: pos and vel (n x 3, updated in place), q (n), inv_mass (n, or NULL for unit mass),
 * forces (n x 3, holds the last step's forces). Positions may leave the cell (every stage wraps them).
 * When ev_steps (DEVICE, steps x 15 doubles) is not NULL, step s stores (E_rec, virial_rec[6], E_real,
 * E_self, virial_real[6]) at ev_steps + 15 s (the real-space part zero without rs). Units as for
 * pme_compute (dt in units where F * inv_mass * dt is a velocity in A per time unit). Chunks of up to 32
 * steps are recorded once as one CUDA graph and replayed, so the host only enqueues; the call returns
 * without waiting: pme_sync(plan) waits and reports device-side errors. rs must use the plan's device; its
 * own stream is not used here. Results equal the same steps driven from the host bit for bit. */
pme_status pme_run_steps(pme_plan *plan, pme_real *rs, float *pos, float *vel, const float *q, const float *inv_mass,
                         int64_t n, float *forces, double dt, int steps, double *ev_steps);

/* ------------------------------------------------------------------------------------------------------ */
/* Batched evaluation: many independent systems per call, replayed from one CUDA graph                      */

/* Paper: Sec. V-C runs several CS / FI pipelines per board and across boards (configurations 1_1 to 4_2)
 * and reports time against problem size in atoms; on one GPU the counterpart is evaluating many
 * independent systems of different sizes together, so that the device stays full. */
/* Build a batch over nsys existing plans (not owned by the batch; each must outlive it and must not be
 * used elsewhere while the batch runs). All plans must use the same B-spline order p. Atom counts n[s] are
 * fixed for the batch. Atom arrays of all systems are packed back to back in the order given: system s owns
 * atoms [off_s, off_s + n[s]) with off_s = n[0] + ... + n[s-1]. Systems of one mesh shape are evaluated
 * together (one launch per stage for the whole group), the groups concurrently; the batch runs on
 * cuda_stream and records its work as one CUDA graph, re-recorded when the array pointers change. Results
 * equal each system's single-system evaluation bit for bit. */
pme_status pme_batch_create(int nsys, pme_plan *const *plans, const int64_t *n, void *cuda_stream, pme_batch **out);

/* Paper: Sec. III-A per system, as for pme_compute; the batch analogue of pme_enqueue. */
/* Evaluate every system of the batch: pos (Ntot x 3), q (Ntot), forces (Ntot x 3) are packed device
 * arrays; ev_dev is a DEVICE array of nsys x 7 doubles (energy, virial[6] per system). Asynchronous:
 * call pme_batch_sync() to wait and collect device-side errors. */
pme_status pme_batch_enqueue(pme_batch *batch, const float *pos, const float *q, float *forces, double *ev_dev);
/* Wait for the batch's stream and return (and clear) any device-side error of the last evaluation. Paper:
 * Sec. III (result collection). */
pme_status pme_batch_sync(pme_batch *batch);

/* How a batch runs its systems. PME_BATCH_GROUPED: systems of one mesh shape share one launch per stage,
 * the shapes' launch chains run as parallel branches of the batch's graph. PME_BATCH_PERSISTENT: one
 * persistent kernel takes (system, stage, item range) entries from a work list in order, each entry
 * waiting (bounded, PME_ETIMEOUT past 1 s) only for its own system's previous stage, so the stages of
 * different systems overlap. PME_BATCH_AUTO (the default): the grouped chains where the systems allow
 * them. Every strategy gives each system its single-system result bit for bit. Takes effect at the next
 * pme_batch_enqueue (which then re-records the graph). Returns PME_EUNSUPPORTED for PME_BATCH_GROUPED
 * when a plan uses 16^3 spreading tiles. Paper: Sec. V-C (several pipelines at once); the work list is
 * this library's own scheduling. */
enum { PME_BATCH_AUTO = 0, PME_BATCH_GROUPED = 1, PME_BATCH_PERSISTENT = 2 };
pme_status pme_batch_set_strategy(pme_batch *batch, int strategy);
/* Tune a batch on its own packed DEVICE arrays (as for pme_batch_enqueue): the grouped strategy with every
 * plan's spread / force CTA size at 128, 256 and the density rule, and the persistent strategy, each timed
 * over reps evaluations after a bit-for-bit comparison with the first; the fastest identical one is kept
 * (plans are set to 8^3 tiles, which grouped launches need). *strategy and *us_per_batch (host, either may
 * be NULL) report the choice. Synchronous. */
pme_status pme_batch_autotune(pme_batch *batch, const float *pos, const float *q, float *forces, double *ev_dev,
                              int reps, int *strategy, double *us_per_batch);

/* The strategy the next pme_batch_enqueue uses (PME_BATCH_GROUPED or PME_BATCH_PERSISTENT), or -1 for a
 * NULL batch. */
int pme_batch_get_strategy(const pme_batch *batch);
/* Releases the batch's own state (not its plans). The batch must be idle. */
void pme_batch_destroy(pme_batch *batch);

/* ------------------------------------------------------------------------------------------------------ */
/* Serving: continuous batching of independent requests                                                   */

/* The paper has no serving counterpart: this request loop is an interface of the library for callers that
 * submit independent evaluations (different systems, different atom counts and meshes) as they arrive. */
/* A server owns a worker thread that admits submitted requests into "waves" (requests of one mesh shape
 * share one launch per stage) while earlier waves are still running, bounded by max_slots requests in
 * flight and by mem_budget_bytes of device memory held by the plans of in-flight requests. */
pme_status pme_server_create(size_t mem_budget_bytes, int max_slots, pme_server **out);

/* No counterpart in the paper (serving interface); each request is one Sec. III-A evaluation. */
/* Submit one evaluation on a resident plan. pos, q, forces are device arrays that must stay valid until
 * pme_poll returns PME_OK or an error; energy (double*) and virial (double[6]) are host pointers written
 * before completion is reported (either may be NULL). Requests on the same plan run one at a time, in
 * submission order. Returns PME_EAGAIN when max_slots requests are already queued or in flight, or the
 * plan alone exceeds the memory budget (PME_ENOMEM). */
pme_status pme_submit(pme_server *srv, pme_plan *plan, const float *pos, const float *q, int64_t n, float *forces,
                      double *energy, double *virial, pme_ticket *out);

/* No counterpart in the paper (serving interface). */
/* Query a ticket: PME_OK when done (results written; the ticket is then retired), PME_PENDING while in
 * flight, or the request's error. block != 0 waits until it is done. */
pme_status pme_poll(pme_server *srv, pme_ticket ticket, int block);

/* No counterpart in the paper (serving interface). */
/* Device-side latency statistics of completed requests (microseconds from submit to completion). */
pme_status pme_server_stats(pme_server *srv, int64_t *completed, double *p50_us, double *p99_us, int64_t *waves);

/* Stops the worker after the requests in flight complete and releases the server. */
void pme_server_destroy(pme_server *srv);

/* ------------------------------------------------------------------------------------------------------ */
/* Errors and test hooks                                                                                   */

/* No counterpart in the paper: error reporting of this library. Static text for a status code. */
const char *pme_strerror(pme_status s);

/* No counterpart in the paper: error reporting of this library. */
/* Copy the calling thread's last error message (NUL-terminated, truncated to len) into buf. Returns the
 * status that produced it (PME_OK if none). */
pme_status pme_last_error_detail(char *buf, size_t len);

/* No counterpart in the paper: failure injection for tests of this library. When nth > 0, the nth
 * allocation the library makes from now on (a host object, device memory or page-locked host memory; every
 * entry point counts) fails as if the system were out of memory, and the call that made it returns
 * PME_ENOMEM after releasing what it had allocated; nth = 0 disarms. Process-wide. */
pme_status pme_debug_fail_alloc(int nth);

/* No counterpart in the paper: a throughput probe of the resource the charge-spreading step (Sec. III-A
 * "Charge Spreading") is bound by on this GPU, for stating its achieved rate against a measured peak.
 * Enqueues one probe kernel of ctas CTAs on cuda_stream and returns in *ops the number of operations it
 * performs (time it with events on that stream): kind 0 = conflict-free shared-memory 32-bit integer
 * atomicAdd (buf: DEVICE, at least 4 bytes per CTA, receives a checksum per CTA); kind 1 = 64-bit integer
 * reductions into global memory spread over buf (DEVICE, buf_bytes, keep it L2-sized; its contents are
 * incremented). Returns PME_EINVAL for other kinds, sizes or NULL pointers. */
pme_status pme_probe_launch(int kind, int ctas, int rounds, void *buf, size_t buf_bytes, void *cuda_stream,
                            double *ops);

/* No counterpart in the paper: failure detection of this library (a bounded device-side wait that gives
 * up and reports, instead of hanging). */
/* Test hook: when set (nonzero) on a batch, the batch runs as one persistent work-list kernel whose
 * entries wait (bounded) for their dependencies, and its next launch makes one such wait on a counter that
 * nothing advances. The bounded wait gives up after wait_limit_ns (<= 2 s) and the launch reports
 * PME_ETIMEOUT from pme_batch_sync(), leaving the device usable. 0 restores normal operation. */
pme_status pme_batch_debug_stall(pme_batch *batch, int enable, int64_t wait_limit_ns);

#ifdef __cplusplus
}
#endif

#endif /* PME_GB300_H */
