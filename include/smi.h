/*
 * smi.h -- C ABI of the GB300 staggered-grid acoustic modelling / RTM /
 * FWI-gradient library (libsmi.so, CUDA, sm_103a).
 *
 * Method: SMIwiz, arXiv 2311.02293.  The library computes, on one GPU:
 *   smi_forward      seismograms of the first-order acoustic system
 *                    (Sec. 2.1, Eq. acoustic and its leap-frog update
 *                    equations) with CPML layers, Kaiser-sinc source
 *                    injection / receiver extraction and the dynamic
 *                    computing box (Sec. 4.1);
 *   smi_rtm          the zero-lag cross-correlation image (Sec. 2.3,
 *                    Eq. rtmimage), the observed data back-propagated as
 *                    the adjoint source;
 *   smi_fwi_gradient the least-squares misfit (Eq. objfwi) and its exact
 *                    discrete gradient with respect to Vp (Eq.
 *                    gradrhokappa via kappa = rho Vp^2), Algorithm 2, with
 *                    the source field rebuilt backwards from saved
 *                    boundaries (Sec. 4.2; every dr-th step stored and
 *                    interpolated in time with a Kaiser-windowed sinc of
 *                    radius 8 samples when dr > 1).
 *
 * Conventions
 *   - Axes: n1 = z (fastest), n2 = x, n3 = y (Sec. 3.6).  A 2D model has
 *     n3 = 1.  Model arrays hold n1*n2*n3 floats, z fastest.
 *   - Positions: metres (z, x, y) from the first physical node (Sec. 3.4).
 *     A position within 1e-6 cells of a node uses that node alone; other
 *     positions use the Kaiser-windowed sinc of radius order/2 (Sec. 3.8).
 *   - Seismograms: for shot s, nt x nrec_s floats (receiver fastest) at
 *     offset nt * rec_offset[s]; sample it holds p at time (it+1) dt.
 *   - The extended grid adds nb CPML layers on every face; the model is
 *     extended into them by copying the nearest physical value.
 *
 * Pointers
 *   Model arrays, the wavelet, observed data and every output may be host
 *   or device pointers (the library asks the CUDA runtime which); geometry
 *   arrays are always host pointers.  The caller owns all of them.  The
 *   library allocates its working state (wavefields, CPML slabs, saved
 *   boundaries, tables) on the device with stream-ordered allocations on
 *   opts->stream and frees it before returning.
 *
 * Calls are blocking: each returns after its work on opts->stream has
 * finished.  Calls on different streams from different host threads may
 * run concurrently on the GPU.
 *
 * Errors: every int-returning call returns SMI_OK (0) or a negative
 * SMI_ERR_* code and records a message readable with smi_last_error() on
 * the calling thread.  No call exits the process.
 */
#ifndef SMI_H
#define SMI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SMI_OK 0
#define SMI_ERR_ARG (-1)          /* bad size, option, pointer or position */
#define SMI_ERR_CFL (-2)          /* Eq. cfl violated (Sec. 3.8: the paper stops) */
#define SMI_ERR_DISPERSION (-3)   /* too few points per wavelength (Sec. 3.8) */
#define SMI_ERR_NOMEM (-4)        /* device allocation failed / over budget */
#define SMI_ERR_UNSTABLE (-5)     /* a non-finite value appeared */
#define SMI_ERR_TIMEOUT (-6)      /* a bounded device wait gave up */
#define SMI_ERR_CUDA (-7)         /* a CUDA runtime call failed */
#define SMI_ERR_UNSUPPORTED (-8)  /* a size the library does not support (boundary bands of a step >= 2^31 values) */

/* Kernel family (smi_opts.kernels).  Every family computes the same scheme;
 * results agree to FP32 rounding. */
#define SMI_KERNELS_AUTO 0        /* the fastest measured kernels that support the problem: in 3D the two-pass
                                     tile kernels (a velocity pass, then a pressure pass) with the z / x CPML
                                     terms in band kernels over the slabs, in 2D the 2D tile kernels */
#define SMI_KERNELS_GENERIC 1     /* the generic grid-stride kernels (CPML inline, 64-bit indexing) that
                                     serve 3D fields of 2^31 points or more and smi_forward_noalloc; for
                                     tests that check them against the oracle on small problems */
#define SMI_KERNELS_TWOPASS 2     /* 3D: the two-pass tile kernels with the CPML band kernels (what AUTO runs) */
#define SMI_KERNELS_FUSED 3       /* 3D forward and adjoint steps: the single-pass kernel (velocity and pressure
                                     in one pass, CPML of all axes inline, state double buffered); no free
                                     surface (falls back to two-pass).  Measured slower than AUTO on GB300 */
#define SMI_KERNELS_INLINE 4      /* 3D forward and adjoint steps: the two-pass tile kernels launched as an
                                     interior and a CPML-band tile class, the z / x CPML terms inline in the
                                     band class (no band kernels).  Measured slower than AUTO on GB300 */

/* Storage precision of the saved boundaries (Sec. 4.2). */
#define SMI_PREC_F32 0
#define SMI_PREC_F16 1            /* FP16 with one FP32 scale per step, face and axis */
#define SMI_PREC_BF16 2           /* BF16 with the same scaling */

/* Velocity model (Secs. 2.1, 3.5, 3.6).  vp, rho: n1*n2*n3 floats, z
 * fastest, host or device, strictly positive.  kappa = rho vp^2. */
typedef struct {
    int ndim;                 /* 2 or 3 */
    int n1, n2, n3;           /* physical sizes z, x, y (n3 = 1 in 2D) */
    double d1, d2, d3;        /* grid spacings in metres (d3 unused in 2D) */
    const float *vp;
    const float *rho;
} smi_model;

/* Acquisition (Sec. 3.4): one pressure source per shot and its receivers,
 * stored like the paper's acquisition file (z, x, y per line) in CSR form.
 * All host pointers. */
typedef struct {
    int nshot;
    const double *src;        /* [nshot][3] source position (z, x, y) in metres */
    const int *rec_offset;    /* [nshot + 1] receivers of shot s: rec_offset[s] .. rec_offset[s+1]-1 */
    const double *rec;        /* [rec_offset[nshot]][3] receiver positions */
} smi_geometry;

/* Source time function (Sec. 3.5): nt samples, stf[it] applied at step it
 * as p += dt * stf[it] * w / dV over the source stencil.  Host or device. */
typedef struct {
    int nt;                   /* time steps */
    double dt;                /* time step (s) */
    double fm;                /* centre frequency (Hz): CPML alpha and the dispersion check */
    const float *stf;
} smi_wavelet;

/* Scheme options (Secs. 3.6, 3.8, 4.1, 4.2).  Fill with smi_opts_default(). */
typedef struct {
    int order;                /* 4 or 8 (FD order in space, Sec. 3.8) */
    int nb;                   /* CPML layers per face, >= order/2 (paper: 20) */
    int freesurf;             /* 1: free surface on the top face by the image method (Sec. 2.1): p = 0
                                 at the first physical node row, p mirrored antisymmetrically and v_z
                                 symmetrically into the top layer (which then absorbs nothing);
                                 source / receiver weights above the surface fold, negated, onto
                                 their mirror nodes.  0: absorbing top face.  Else SMI_ERR_ARG */
    int dr;                   /* boundary decimation ratio (Sec. 4.2): the boundary of every dr-th
                                 step is stored and interpolated in time during reconstruction;
                                 1 <= dr <= 5 vmax / vmin (SMI_ERR_ARG otherwise) */
    int use_box;              /* dynamic computing box (Sec. 4.1), 1 = on */
    int shell_prec;           /* SMI_PREC_* storage of the saved boundaries */
    double kaiser_b;          /* Kaiser window shape (default 4.0) */
    double cpml_R;            /* CPML target reflection (default 1e-3; 1 = no absorption) */
    void *stream;             /* cudaStream_t to run on; NULL = the legacy default stream */
    int max_batch;            /* shots propagated together in one launch; 0 = automatic */
    int profile;              /* 1: time the stencil kernels with CUDA events (smi_last_stats) */
    int img_norm;             /* smi_rtm only: 0 the zero-lag cross-correlation (Eq. rtmimage); 1 each
                                 shot's image divided by its source illumination sum_t p_s^2 + eps,
                                 eps = 1e-3 of the shot's largest illumination (Sec. 2.3) */
    int kernels;              /* SMI_KERNELS_AUTO (default), _GENERIC, _TWOPASS, _FUSED or _INLINE; else
                                 SMI_ERR_ARG */
    int per_shot;             /* 1: smi_rtm and smi_fwi_gradient return each shot's result instead of the sum
                                 over shots: image / gradient [nshot][n3][n2][n1] and misfit [nshot],
                                 shot s equal to a call with shot s alone (the shots of a batch share
                                 launches).  Not with img_norm, the family gradients or the tape calls
                                 (SMI_ERR_ARG); no effect on smi_forward.  0: sums (default) */
} smi_opts;

/* Per-call measurements, filled for the calling thread's last call.  Index
 * 0 = forward stencil steps, 1 = adjoint stencil steps, 2 = source-field
 * reconstruction steps (with the fused imaging / gradient accumulation). */
typedef struct {
    double point_updates;     /* grid points advanced one step, summed over all propagations */
    double bytes[3];          /* algorithmic HBM bytes of those steps (FP32: 40 B per 3D point,
                                 32 B per 2D point, +16 B per CPML axis at slab points;
                                 reconstruction 52 B (3D) / 44 B (2D) with the accumulator) */
    double ms[3];             /* summed CUDA-event time of those steps (opts.profile = 1) */
    long long steps[3];       /* stencil steps taken (per shot) */
    long long kernel_launches;   /* every kernel the call launched */
    double device_bytes;      /* peak device memory the call allocated: set-up tables plus its largest
                                 batch of shots (fields, saved boundaries, accumulators) */
    long long band_values;    /* boundary values saved per shot per step (0 for forward) */
} smi_stats;

/* Fills *o with: order 4, nb 20, freesurf 0, dr 1, use_box 1, FP32
 * boundaries, kaiser_b 4.0, cpml_R 1e-3, default stream, automatic batch,
 * no profiling. */
void smi_opts_default(smi_opts *o);

/* Forward modelling, Algorithm 2 forward loop (Sec. 2.1; box Sec. 4.1).
 * seis: sum_s nt*nrec_s floats (layout above), host or device, written. */
int smi_forward(const smi_model *model, const smi_geometry *geom, const smi_wavelet *wav,
                const smi_opts *opts, float *seis);

/* RTM image, Eq. rtmimage with the observed data as adjoint source
 * (Sec. 2.3; Algorithm 2).  dobs: observed seismograms (seis layout).
 * image: n1*n2*n3 floats, written with sum_s sum_it kappa*pbar * p at equal
 * time levels, pbar being the exact discrete adjoint field. */
int smi_rtm(const smi_model *model, const smi_geometry *geom, const smi_wavelet *wav,
            const smi_opts *opts, const float *dobs, float *image);

/* FWI misfit J = 1/2 sum (u - d)^2 over shots, receivers and samples
 * (Eq. objfwi) and its gradient with respect to Vp on the physical grid
 * (Eq. gradrhokappa, exact for the discrete scheme, CPML-layer model held
 * fixed), Algorithm 2.  misfit: one double, host or device.  grad_vp:
 * n1*n2*n3 floats, host or device.  Either may be NULL. */
int smi_fwi_gradient(const smi_model *model, const smi_geometry *geom, const smi_wavelet *wav,
                     const smi_opts *opts, const float *dobs, double *misfit, float *grad_vp);

/* FWI misfit (as smi_fwi_gradient) and its gradient in a parametrisation
 * family (Sec. 2.2: family 1 = (Vp, rho), family 2 = (Vp, Ip) with
 * Ip = rho Vp), from both parts of Eq. gradrhokappa by the chain rule:
 *   dJ/dVp|rho = 2 rho Vp dJ/dkappa,   dJ/drho|Vp = Vp^2 dJ/dkappa + dJ/drho|kappa,
 *   family 2:  dJ/dVp|Ip = dJ/dVp|rho - dJ/drho|Vp rho / Vp,  dJ/dIp = dJ/drho|Vp / Vp.
 * dJ/drho|kappa is the exact discrete gradient through the half-node
 * buoyancy 2 / (rho_i + rho_{i+1}); the CPML cells' rho and kappa are held
 * fixed.  log_param = 1: gradients with respect to the logarithms of the
 * parameters (each multiplied by its parameter), the log transform of
 * Sec. 3.7.  grad1 (Vp), grad2 (rho or Ip): n1*n2*n3 floats each, host or
 * device, both required; misfit may be NULL.  family outside {1, 2} or
 * log_param outside {0, 1}: SMI_ERR_ARG.  Costs one extra set of source
 * velocities per shot of a batch and one accumulator per axis. */
int smi_fwi_gradient_family(const smi_model *model, const smi_geometry *geom, const smi_wavelet *wav,
                            const smi_opts *opts, const float *dobs, int family, int log_param, double *misfit,
                            float *grad1, float *grad2);

/* Vector-Jacobian product of smi_forward with respect to Vp: for an upstream
 * gradient g = dL/dseis (adj_src, seis layout, host or device), writes
 * dL/dVp = sum over shots, receivers and samples of g * d seis / d Vp on the
 * physical grid (grad_vp, n1*n2*n3 floats, host or device).  It is the FWI
 * gradient computation (Eq. gradrhokappa, Algorithm 2) with g in place of
 * the residual: forward modelling saving the boundaries (Sec. 4.2), then the
 * exact discrete adjoint with g as its source.  The saved boundaries are the
 * checkpoint; no wavefield history is kept. */
int smi_forward_vjp(const smi_model *model, const smi_geometry *geom, const smi_wavelet *wav,
                    const smi_opts *opts, const float *adj_src, float *grad_vp);

/* Forward modelling that keeps its checkpoint for one later reverse pass
 * (the boundary-saving strategy of Sec. 4.2 as the checkpoint of automatic
 * differentiation): writes the seismograms like smi_forward and returns in
 * *tape the saved boundaries (every dr-th step, opts->shell_prec storage),
 * the wavefield state after the last step and the set-up tables, all on the
 * device, for every shot at once (SMI_ERR_NOMEM if they do not fit).
 * smi_tape_vjp then runs only the reverse loop (adjoint, source-field
 * reconstruction, gradient accumulation): three modellings per gradient in
 * all instead of the four of smi_forward followed by smi_forward_vjp.  The
 * model, wavelet and stream arrays the call read must stay valid until
 * smi_tape_free.  On error *tape is NULL. */
typedef struct smi_tape smi_tape;
int smi_forward_tape(const smi_model *model, const smi_geometry *geom, const smi_wavelet *wav,
                     const smi_opts *opts, float *seis, smi_tape **tape);

/* dL/dVp (grad_vp, n1*n2*n3 floats, host or device) for the upstream
 * gradient adj_src = dL/dseis (seis layout, host or device) of the
 * smi_forward_tape call that made the tape, exactly as smi_forward_vjp
 * computes it, without a forward run.  stream: cudaStream_t or NULL.  A tape
 * serves one reverse pass (the pass consumes the kept state): a second call
 * returns SMI_ERR_ARG. */
int smi_tape_vjp(smi_tape *tape, const float *adj_src, float *grad_vp, void *stream);

/* Frees a tape's device memory (synchronising with the device); NULL is a
 * no-op. */
void smi_tape_free(smi_tape *tape);

/* Adjoint of the forward map with respect to the wavelet (the transpose of
 * smi_forward as a linear map stf -> seismograms, Eq. adj of Sec. 2.2 with
 * the source term's adjoint read at the source): for adj_src d (seis layout,
 * host or device) writes stf_adj[it] = sum over shots of the exact discrete
 * adjoint pressure sampled with the source stencil, times dt / dV (nt floats,
 * host or device).  Runs the adjoint propagation only (no forward run, no
 * boundaries); the adjoint box (Sec. 4.1) is the receivers' box as in
 * smi_fwi_gradient.  The dot-product identity <L f, d> = <f, L^T d> checks
 * it against smi_forward.  wav->stf is validated but not read. */
int smi_forward_adjoint(const smi_model *model, const smi_geometry *geom, const smi_wavelet *wav,
                        const smi_opts *opts, const float *adj_src, float *stf_adj);

/* FP64 inner product of two float arrays of n elements on the device (the
 * reduction of the dot-product test and of misfits, Eq. objfwi): products
 * and sums in FP64, partial sums added in a fixed order, so the result does
 * not depend on scheduling.  a, b: device arrays of the current device
 * (SMI_ERR_ARG otherwise); out: one double, host or device.  stream:
 * cudaStream_t or NULL.  Blocking. */
int smi_dot(const float *a, const float *b, size_t n, double *out, void *stream);

/* Sizes a caller needs before a call: seismogram floats, image floats and
 * the device bytes the call will allocate (kind: 0 forward, 1 rtm, 2
 * gradient, 3 vector-Jacobian product, 4 gradient of a parametrisation
 * family).  Validates like the calls themselves (CFL, dispersion,
 * positions) and launches one small reduction to find vmin/vmax.  Any
 * output pointer may be NULL. */
int smi_query(const smi_model *model, const smi_geometry *geom, const smi_wavelet *wav,
              const smi_opts *opts, int kind, size_t *seis_elems, size_t *image_elems,
              size_t *device_bytes);

/* The device bytes of a call (smi_query's device_bytes, estimated the same
 * way) from the sizes alone: no device work and no wait on the GPU, for
 * admission decisions while other work runs.  Checks the arguments
 * (SMI_ERR_ARG) but not CFL, dispersion or positions: a call that fails
 * those fails when it runs. */
int smi_footprint(const smi_model *model, const smi_geometry *geom, const smi_wavelet *wav,
                  const smi_opts *opts, int kind, size_t *device_bytes);

/* Computing-box bounds (Sec. 4.1) as the kernels compute them on the
 * device: for shot `shot`, the box around its source (which = 0) or its
 * receivers (which = 1) after n = n0 .. n0+count-1 steps.  lo, hi: host
 * [count][3] ints, inclusive extended-grid indices in axis order z, x, y;
 * an empty box has hi < lo. */
int smi_box_table(const smi_model *model, const smi_geometry *geom, const smi_wavelet *wav,
                  const smi_opts *opts, int shot, int which, int n0, int count, int *lo, int *hi);

/* Forward modelling that allocates no device memory, for callers that may
 * not call cudaMalloc: code running where another runtime or a caching
 * allocator already owns the device's memory, or loops that cannot afford an
 * allocation's synchronisation or failure.  The paper has no counterpart; it
 * computes exactly what smi_forward computes.
 *   - Working memory is one fixed 64 MiB device array inside the library
 *     (resident on every GPU that loads the library until the process
 *     exits).  A problem needs about 4*(ndim+3) bytes per extended grid
 *     node plus CPML and stencil tables; larger problems, or an axis of more
 *     than 8192 extended nodes, return SMI_ERR_ARG with the size needed.
 *   - vp, rho, stf and seis must be device pointers (SMI_ERR_ARG otherwise);
 *     geometry stays on the host.  Shots run one after another.
 *   - The first call on a device looks up the array's device address; make
 *     that first call before any stream capture.
 *   - All calls share the array: calls that overlap on the GPU (other
 *     streams, other host threads) race and corrupt each other's results.
 *     The array keeps the last call's contents; every shot clears what must
 *     start at zero. */
int smi_forward_noalloc(const smi_model *model, const smi_geometry *geom,
                        const smi_wavelet *wav, const smi_opts *opts, float *seis);

/* ---------------------------------------------------------------------------
 * Request server (continuous batching of modelling jobs on one GPU).  The
 * GPU counterpart of the paper's shot-per-process parallelism (Sec. 3.2) and
 * batchwise job scheduling (Sec. 4.3): requests of any size, dimension and
 * nt are queued in arrival order and admitted into one of `slots` worker
 * slots (each with its own CUDA stream and host thread) as soon as a slot is
 * free and the request's device footprint (smi_query) fits in the remaining
 * memory budget; admitted requests run concurrently.  Among queued requests
 * the oldest one that fits is admitted first.  A request's footprint comes
 * from smi_footprint (no device work at submission); a request whose
 * footprint exceeds the whole budget fails at submission with SMI_ERR_NOMEM.
 * Single-shot requests of one survey -- same kind (forward, RTM without
 * img_norm, gradient), the same model arrays (vp, rho pointers), wavelet
 * (stf pointer, nt, dt, fm) and options -- that are queued when a slot admits
 * the first of them join its call, up to 64 shots while they fit the budget
 * and their extended grids sum to at most 2^24 points (one launch over them
 * would not yet fill the GPU; a 300^3 shot joins none):
 * one shot-batched call whose shots share every launch, with per-shot results
 * (opts.per_shot) copied back to each request's own outputs.  Each request's
 * result equals the same request run alone.  If a merged call fails (a
 * request invalid on its own: a position outside the model, CFL), its
 * requests run one by one, so that only the invalid one reports the error. */
typedef struct smi_server smi_server;

typedef struct {
    int kind;                 /* 0 forward (out = seismograms), 1 RTM (out = image),
                                 2 FWI gradient (out = grad_vp, misfit) */
    smi_model model;
    smi_geometry geom;
    smi_wavelet wav;
    smi_opts opts;            /* opts.stream is replaced by the slot's stream */
    const float *dobs;        /* observed data (kinds 1, 2) */
    float *out;               /* output array, as for the direct calls */
    double *misfit;           /* kind 2, may be NULL */
} smi_request;                /* every pointer stays owned by the caller and must
                                 stay valid until the request has finished */

typedef struct {
    int status;               /* SMI_OK or the request's SMI_ERR_* code */
    size_t device_bytes;      /* admitted footprint */
    double t_submit, t_start, t_end;   /* seconds since the server was created */
    char error[256];
} smi_result;

/* budget_bytes = 0: 80 % of the device's free memory at creation.  The
 * device current at creation runs every request of the server. */
smi_server *smi_server_create(size_t budget_bytes, int slots);
/* Queues *req (copied); *ticket identifies it.  Returns SMI_ERR_ARG only for
 * a malformed call; request errors are reported by smi_wait. */
int smi_submit(smi_server *s, const smi_request *req, long long *ticket);
/* Waits for the request to finish (timeout_s < 0: no limit); SMI_ERR_TIMEOUT
 * if it is still queued or running after timeout_s.  Once it has returned a
 * finished request's result, the ticket is released (the server keeps no
 * record of it): later calls with that ticket return SMI_ERR_ARG. */
int smi_wait(smi_server *s, long long ticket, double timeout_s, smi_result *res);
/* *state: 0 queued, 1 running, 2 finished. */
int smi_poll(smi_server *s, long long ticket, int *state);
/* Removes a request that has not started yet (its status becomes SMI_ERR_ARG). */
int smi_cancel(smi_server *s, long long ticket);
int smi_server_info(smi_server *s, size_t *budget, size_t *in_use, long long *queued,
                    long long *completed, long long *failed);
/* Finishes running requests, drops queued ones, joins the workers. */
/* Merged calls the server has made and the requests they carried (each
 * merged call carries two or more). */
int smi_server_merges(smi_server *s, long long *calls, long long *requests);
void smi_server_destroy(smi_server *s);

/* Failure detection (no paper counterpart): exercises the give-up path of
 * the bounded waits that the 3D tile kernels use for their tile copies.  One
 * warp waits, with the kernels' own wait helper, on a barrier that nothing
 * completes; after `polls` polls (polls < 0: the kernels' own limit) it
 * records the give-up and returns, as a tile kernel would before the call
 * reports SMI_ERR_TIMEOUT.  Returns SMI_ERR_TIMEOUT when the wait gave up (the
 * expected outcome; the context stays usable), SMI_OK if the barrier
 * completed, another SMI_ERR_* on a CUDA failure.  ms (may be NULL): the
 * kernel's duration.  stream: cudaStream_t or NULL. */
int smi_wait_check(void *stream, long long polls, double *ms);

/* Measurements of the calling thread's last smi_forward / smi_rtm /
 * smi_fwi_gradient call. */
int smi_last_stats(smi_stats *st);

/* Message of the calling thread's last error ("" after success). */
const char *smi_last_error(void);

/* Library version and target, e.g. "smi 0.1 sm_103a". */
const char *smi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SMI_H */
