/*
 * pim.h -- C ABI of the GB300 FFT-PIM library (libpim.so).
 *
 * FFT periodic interpolation method of Ai & Lomakin, arXiv 2312.02376:
 * the periodic scalar potential
 *
 *     u(r_m) = sum_n G^p(r_m - r_n) q_n                         (Eq. 1)
 *     G^p(r) = sum_i exp(-j k0.(i o L)) G0(r - i o L),
 *     G0(r)  = exp(-j k |r|) / (4 pi |r|)                       (Eq. 2)
 *
 * at N points that are both sources and observers in one cell of a 1D, 2D
 * or 3D periodic array (Sec. 2), evaluated as u = u_near + u_far (Eq. 4-5):
 * the near zone (images |i_d| <= i_d) by Lagrange anterpolation onto a
 * uniform grid, a zero-padded FFT convolution with the tabulated near-zone
 * kernel, interpolation back to the points and a sparse near-pair
 * correction (Sec. 3.3, steps 1-4, Eq. er); the far zone (all other images)
 * by projection onto a sparse grid, a grid-to-grid sum with the series form
 * of the periodic Green's function (Eq. pgf; Eq. lgf in the neutral static
 * case) and interpolation from a grid shifted by half a step (Sec. 3.2,
 * Eq. grid, projection, 8, interpolation).
 *
 * Conventions
 *   - The paper's engineering convention: j = sqrt(-1), time factor e^{jwt},
 *     so the Bloch condition is u(r + a) = exp(-j k0.a) u(r) for a lattice
 *     vector a (the physics form exp(i k0.a) with i = -j).
 *   - The self term n = m is dropped only for the image i = 0; self images
 *     (n = m, i != 0) are kept.
 *   - Complex data are interleaved (re, im).  q and u are [N][nrhs], the
 *     right-hand-side index fastest.  PIM_FP64 plans use complex128 data,
 *     PIM_FP32_MIXED plans complex64.  In the neutral static case
 *     (k = 0 and k0 = 0) the data are real (float64 / float32).
 *   - Pointers may be device or host memory; host buffers are staged
 *     through the plan's device buffers on the given stream (the call then
 *     returns after the result has been copied back).
 *   - Threading: a plan is not thread safe.  All device work of a call is
 *     ordered on the stream passed to that call (0 = the legacy default
 *     stream); the plan's internal streams (far zone, list-free correction)
 *     fork from it and are joined back to it.
 *
 * Errors are returned as pim_status codes; no call aborts the process, and
 * no device fault is used for control flow.  Device-side conditions (a
 * non-neutral input in the neutral static case, an internal bounds check)
 * set a flag that pim_last_device_status() reads after synchronising.
 */
#ifndef PIM_H
#define PIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pim_plan_s* pim_plan;

typedef enum {
    PIM_OK = 0,
    PIM_ERR_ARG = 1,          /* invalid argument (null pointer, size, grid) */
    PIM_ERR_UNSUPPORTED = 2,  /* non-rectangular lattice, p out of range, a complex k or k0
                                 with with_gradient, a 1D complex series outside its
                                 evaluated regimes (k0_imag)                             */
    PIM_ERR_ANOMALY = 3,      /* Rayleigh-Wood anomaly: k_z or k_rho of a Floquet mode ~ 0 (Sec. 2) */
    PIM_ERR_NOT_NEUTRAL = 4,  /* k = k0 = 0 and |sum q| > neutral_tol * sum |q| (Eq. neutral) */
    PIM_ERR_OUT_OF_CELL = 5,  /* a point outside the closed cell [0, D] */
    PIM_ERR_STATE = 6,        /* apply before pim_set_points */
    PIM_ERR_OOM = 7,          /* device allocation failed or mem_cap exceeded */
    PIM_ERR_CUDA = 8,         /* a CUDA runtime call failed */
    PIM_ERR_TIMEOUT = 9,      /* a bounded device wait ran out (the tensor-core kernel's
                                 waits for its own matrix products; reported by
                                 pim_last_device_status)                                  */
    PIM_ERR_DEVICE = 10       /* a device-side bounds check tripped */
} pim_status;

typedef enum {
    PIM_FP64 = 0,             /* every stage in FP64 */
    PIM_FP32_MIXED = 1        /* spread, FFT, gather in FP32 / complex64; far series,
                                 far grid sum, near-pair correction and the neutral
                                 regularisation in FP64 */
} pim_precision;

typedef enum {
    PIM_CORR_FP64 = 0,        /* correction values FP64, FP64 accumulation */
    PIM_CORR_DOUBLE_FLOAT = 1,/* values as FP64 split into two floats, compensated
                                 (double-float) accumulation on the FP32 pipes */
    PIM_CORR_FP32 = 2,        /* values rounded to complex64 after the FP64
                                 cancellation, FP32 accumulation */
    PIM_CORR_COMPACT = 3      /* the default.  Each row holds first the entries with
                                 |d| > 2^-corr_split max_row |d|, as FP64 split into an FP32
                                 head and a bf16 tail per component (12 B, relative
                                 rounding <= 2^-33) summed in double-float, then the others
                                 as complex64 (8 B) summed in FP32: every stored value is
                                 within 2^-33 max_row |d| of its FP64 value */
} pim_corr_mode;

typedef struct {
    int far_n[3];        /* far grid nodes per axis; 0 -> max(10, ceil(4 k D_d))      */
    int far_p;           /* far Lagrange degree; -1 -> p                               */
    int corr_radius;     /* b, error-correction radius D^ER in grid steps; -1 -> p+1   */
    int corr_cube;       /* 0: boxes within D^ER of the observer box (|r - r_m| <=
                            D^ER, Sec. 3.3 step 4); 1: Chebyshev box distance <= b     */
    int corr_mode;       /* pim_corr_mode; ignored (FP64) for PIM_FP64 plans           */
    double neutral_tol;  /* tau of the neutrality check; default 1e-6                  */
    double series_tol;   /* relative truncation of the far series; default 1e-16      */
    size_t mem_cap;      /* bytes; 0 = no cap.  Exceeding it -> PIM_ERR_OOM            */
    int autotune;        /* 1: pim_set_points times the gather kernel's launch shapes
                            and keeps the fastest; 0: default shape                    */
    int with_gradient;   /* 1: pim_set_points also stores the position derivatives of
                            the correction values (48 B per entry, plus 24 B of FP32
                            heads in compact mode), which pim_position_grad needs, and
                            single-RHS applies keep their grid potentials (one more
                            near grid) for pim_position_grad_reuse                   */
    int corr_split;      /* PIM_CORR_COMPACT: the exponent s of the 2^-s max_row |d|
                            threshold above; 0 keeps every entry in the 12-byte form;
                            default 10; 0 <= s <= 30 (else PIM_ERR_ARG)                */
    int gather_variant;  /* -1: launch shape of the gather kernel chosen by autotune
                            (shape 0 without it); v >= 0 forces shape v, which must be
                            below pim_info.gather_variants (which depends on the
                            precision and correction mode; else pim_set_points
                            returns PIM_ERR_ARG)                                       */
    int corr_listfree;   /* list-free correction (Sec. 3.3 step 4 without a stored
                            list): a box whose points times its correction region's
                            points is at least this value has its correction
                            recomputed by every apply -- the exact kernel summed over
                            the region's points minus the region's grid interaction,
                            formed from the box moments on a local grid -- and keeps
                            no stored entries.  The same operator as the stored list
                            (to rounding).  -1: default (131072: per pair the list-free
                            sum costs about a third of a stored entry's traffic, per
                            box it adds a local convolution worth about 10^5 stored
                            entries); 0: off (every correction stored).  Plans with with_gradient store every
                            correction (the gradient reads the stored derivatives); a
                            correction radius whose local grid exceeds 24 nodes per
                            axis (2b + 2 floor(p/2) + p + 3 > 24) also stores all;
                            and so does a complex wavenumber (k_imag != 0).          */
    double k_imag;       /* imaginary part of k (Sec. 2: a lossy medium has Im k < 0;
                            must be <= 0 and finite); default 0                        */
    double k0_imag[3];   /* imaginary parts of the phase shift (k_x0, k_y0, k_z0), 0 on
                            non-periodic axes; default 0.  With k_imag or k0_imag
                            nonzero the far series are summed in complex arithmetic;
                            the 1D series then evaluates H0^(2) of complex arguments
                            and returns PIM_ERR_UNSUPPORTED for an argument z = krho rho
                            of modulus 6..20 within 0.17 rad of the real axis (a weakly
                            lossy propagating mode); with_gradient plans must have
                            real k and k0 (PIM_ERR_UNSUPPORTED)                      */
    int lf_tensor_cores; /* 1 (default): in FP32 plans the grid part of the list-free
                            correction for the boxes whose stencils are not clamped
                            at a face of the grid runs as one matrix product on the
                            tensor cores (TF32 operands split in hi and lo parts,
                            FP32 accuracy; one right-hand side); 0: CUDA cores       */
} pim_options;

typedef struct {
    int n[3];            /* near grid nodes per axis (spanning [0, D_d])               */
    int nf[3];           /* far grid nodes per axis                                    */
    int p, pf, corr_radius, precision, corr_mode, periodic_mask, near_layers;
    int64_t N;           /* points (0 before pim_set_points)                           */
    int64_t nnz;         /* near-pair correction entries                               */
    size_t device_bytes; /* bytes the plan holds on the device                         */
    double plan_ms;      /* wall time of pim_plan_create                               */
    double points_ms;    /* wall time of the last pim_set_points                       */
    int64_t launches;    /* kernels launched by this plan's applies so far             */
    int gather_variant;  /* launch shape of the gather kernel in use                   */
    int gather_variants; /* launch shapes available to this plan                       */
    int64_t lf_boxes;    /* boxes corrected list-free (corr_listfree)                  */
    int64_t lf_points;   /* points in those boxes                                      */
    int64_t lf_pairs;    /* (observer, source, image) pairs their exact kernel sums per
                            apply (partners in the boxes with moments)                */
    int64_t lf_tc_boxes; /* list-free boxes whose grid part runs on the tensor cores  */
} pim_info;

/* Stages timed by the profiling ring (pim_set_profiling). */
typedef enum {
    PIM_STAGE_PERMUTE = 0,   /* regularise (Eq. neutral) and reorder the sources        */
    PIM_STAGE_SPREAD = 1,    /* near step 1: anterpolation onto the grid                */
    PIM_STAGE_FFT = 2,       /* near step 2: the five pruned FFT passes                 */
    PIM_STAGE_GATHER = 3,    /* near steps 3-4: gather and stored-list correction       */
    PIM_STAGE_FAR = 4,       /* far steps 1-3: projection, grid sum, interpolation
                                (second stream; added to u after the gather)            */
    PIM_STAGE_APPLY = 5,     /* the whole apply, first to last launch                   */
    PIM_STAGE_LF_EXACT = 6,  /* list-free boxes: exact kernel summed over their regions  */
    PIM_STAGE_LF_GRID = 7,   /* list-free boxes: minus the regions' grid interaction    */
    PIM_STAGE_CORR_MULTI = 8,/* several right-hand sides: the one stored-list correction
                                launch for all of them (recorded in the ring slot of the
                                call's last right-hand side)                            */
    PIM_STAGE_LF_TC_GEMM = 9,/* list-free grid part on the tensor cores: the matrix
                                product(s) alone (first to last batch)                  */
    PIM_NUM_STAGES = 10
} pim_stage;

/* Fills *opt with the defaults documented above. */
void pim_options_default(pim_options* opt);

/* Human-readable name of a status code (static string). */
const char* pim_status_string(pim_status s);

/* Message of the last error raised by a call on this thread ("" if none);
 * valid until the next call. */
const char* pim_last_error(void);

/*
 * pim_plan_create -- pre-processing of Sec. 3.2-3.3 that does not depend on
 * the points: near grid, near-zone kernel table (G_near of Eq. 4 on the
 * grid, Sec. 3.3 step 2) and its spectrum on the zero-padded grid, far grids
 * (Eq. grid) and the far table G_far = G^p - G_near (Sec. 3.2) from the
 * series of Eq. pgf / Eq. lgf.
 *
 *   out            receives the plan (NULL on error).
 *   lattice        3x3 row-major, rows a1, a2, a3.  Must be diagonal
 *                  (rectangular cell, PIM_ERR_UNSUPPORTED otherwise).  The
 *                  diagonal gives the cell extents D_d; on periodic axes the
 *                  period is L_d = D_d.
 *   periodic_mask  bit d set: periodic along axis d (0 = free space, near
 *                  zone only).
 *   k              wavenumber (k_0 of the paper), real part, >= 0; its
 *                  imaginary part (a lossy medium, Sec. 2) is opt->k_imag.
 *   k0             phase shift per axis (k_x0, k_y0, k_z0), real parts; must be 0
 *                  on non-periodic axes; imaginary parts in opt->k0_imag.
 *   h              grid spacing per axis: D_d / h_d must be an integer; the
 *                  grid has n_d = D_d / h_d + 1 nodes spanning [0, D_d].
 *   p              near Lagrange degree (p+1 nodes per axis), 2..4.
 *   near_layers    i_d >= 0, near-zone image layers per periodic axis (Eq. 4).
 *   prec           pim_precision.
 *   opt            options (NULL = defaults); copied.
 *   stream         cudaStream_t (NULL = legacy default stream) for the
 *                  table kernels; the call synchronises before returning.
 * Returns PIM_OK, PIM_ERR_ARG, PIM_ERR_UNSUPPORTED, PIM_ERR_ANOMALY,
 * PIM_ERR_OOM or PIM_ERR_CUDA.  The plan owns every device buffer it makes.
 */
pim_status pim_plan_create(pim_plan* out, const double lattice[9], unsigned periodic_mask, double k,
                           const double k0[3], const double h[3], int p, int near_layers,
                           pim_precision prec, const pim_options* opt, void* stream);

/*
 * pim_set_points -- the point-dependent pre-processing (Sec. 3.2 and 3.3):
 * bins the points into the grid's boxes (counting sort), stores their
 * stencils and interpolation coordinates, and builds the near-pair
 * correction list of Sec. 3.3 step 4 (Eq. er, single-extra-image rule) with
 * its values exp(-j k0.(i o L)) [G0(r_m - r_n - i o L) - G_grid] in FP64;
 * for the boxes corrected list-free (opt.corr_listfree) it builds their
 * region tables instead of stored entries.
 *
 *   xyz   N x 3 row-major FP64 positions, device or host pointer; copied.
 *         Every point must lie in the closed cell [0, D] (else
 *         PIM_ERR_OUT_OF_CELL).
 * Replaces the points of an earlier call.  Synchronises before returning.
 */
pim_status pim_set_points(pim_plan plan, int64_t N, const double* xyz);

/*
 * pim_apply -- u = A q (Eq. 1 through Eq. 5): near spread, FFT
 * convolution, gather and correction, plus the far-zone projection, grid
 * sum and interpolation (run on a second stream and joined).
 *   q     [N][nrhs] source strengths in the caller's point order.
 *   u     [N][nrhs] potentials, written (not accumulated).  May not alias q.
 *   nrhs  >= 1.
 * Neutral static plans remove the FP64 mean of q first; a non-neutral q
 * sets the device flag PIM_ERR_NOT_NEUTRAL (see pim_last_device_status).
 * Asynchronous on `stream` for device pointers; synchronous for host ones.
 */
pim_status pim_apply(pim_plan plan, const void* q, void* u, int nrhs, void* stream);

/*
 * pim_apply_adjoint -- w = A^H v, the exact conjugate transpose of the
 * discrete operator of pim_apply (same weights, conjugated spectrum and
 * correction values, far grids with their roles swapped).  Not part of the
 * paper; needed for gradients.  Same layout and semantics as pim_apply.
 * Neutral static plans remove the mean of w (the projector is self-adjoint).
 */
pim_status pim_apply_adjoint(pim_plan plan, const void* v, void* w, int nrhs, void* stream);

/*
 * pim_position_grad -- the gradient of Re sum_{m,r} conj(g[m][r]) u[m][r]
 * with respect to the point positions, u = A q (the same operator as
 * pim_apply), with the discrete structure held fixed ("frozen topology":
 * stencil starts, boxes and correction list as set by pim_set_points):
 *   grad_xyz[k][d] = Re sum_{m,r} conj(g[m][r]) d u[m][r] / d x_{k,d}.
 * With g = dL/du in PyTorch's convention this is dL/dx of a real loss L.
 * It differentiates the Lagrange weights of every interpolation (near
 * and far, observer and source side) and the exact and grid terms of every
 * correction value.  Not part of the paper.
 *   q, g      [N][nrhs], caller order, the plan's data type; device or host.
 *   grad_xyz  N x 3 FP64, caller order, written; device or host.
 * Requires a plan created with opt.with_gradient = 1 (PIM_ERR_STATE
 * otherwise).  Neutral static plans remove the mean of q as pim_apply does.
 */
pim_status pim_position_grad(pim_plan plan, const void* q, const void* g, double* grad_xyz, int nrhs, void* stream);

/*
 * pim_position_grad_reuse -- pim_position_grad for one right-hand side that
 * reuses the near and far grid potentials of the plan's last single-RHS
 * pim_apply (U = K Q(q), u_f) and last single-RHS pim_apply_adjoint
 * (V = K^H Q(g), v_f) instead of recomputing them: the position-gradient
 * kernel alone, after a forward and an adjoint apply (the backward pass of
 * a differentiable apply).  Not part of the paper.
 *   q, g      [N], the very arrays those two applies read (the caller's
 *             guarantee: the plan cannot check their contents); device or host.
 *   grad_xyz  N x 3 FP64, written, as in pim_position_grad.
 * Both applies must have run on a with_gradient plan since the last
 * pim_set_points or pim_update_positions, with no multi-RHS apply,
 * pim_apply_noalloc or pim_position_grad after them (PIM_ERR_STATE
 * otherwise); issue it on their stream or after they completed.
 */
pim_status pim_position_grad_reuse(pim_plan plan, const void* q, const void* g, double* grad_xyz, void* stream);

/*
 * pim_set_points_observers -- sources and observer points apart from them
 * (the paper's accuracy test, Sec. 4.1, evaluates the potential at points
 * that carry no source).  N sources, then M >= 1 observers, each N x 3 / M x 3
 * FP64 (device or host), form the plan's point set in that order (an
 * observer is a point of zero strength); everything pim_set_points does is
 * done for the N + M points, and pim_apply / pim_apply_adjoint act on all of
 * them.  An observer that coincides with a source modulo the lattice is
 * rejected like two coinciding points (PIM_ERR_ARG).  A later pim_set_points
 * drops the observers.
 */
pim_status pim_set_points_observers(pim_plan plan, int64_t N, const double* xyz, int64_t M, const double* obs_xyz);

/*
 * pim_apply_observers -- the potentials at the M observers due to the N
 * sources (Eq. 1 with r_m an observer): u_obs = rows of A at the observers
 * applied to [q; 0].  q [N][nrhs], u_obs [M][nrhs], the plan's data type,
 * device or host (host copies synchronise).  In the neutral static case the
 * regularisation of Eq. neutral removes the mean of q over the sources, and
 * the neutrality test is on q (PIM_ERR_NOT_NEUTRAL via
 * pim_last_device_status).  PIM_ERR_STATE without observers.
 *
 * pim_apply_observers_adjoint -- the adjoint of that map: w [N][nrhs] from
 * v [M][nrhs] (the source rows of A^H applied to [0; v]; in the neutral
 * static case projected on the sources' neutral subspace).
 */
pim_status pim_apply_observers(pim_plan plan, const void* q, void* u_obs, int nrhs, void* stream);
pim_status pim_apply_observers_adjoint(pim_plan plan, const void* v_obs, void* w, int nrhs, void* stream);

/*
 * pim_update_positions -- moves the points of the last pim_set_points to new
 * positions (N x 3 FP64, caller order, device or host) while keeping the
 * discrete structure: the box order, every stencil start, the box of every
 * point and the correction list stay as they were; local coordinates and
 * correction values (and their derivatives, if stored) are recomputed.  For
 * small moves between the steps of a simulation and for finite-difference
 * checks of pim_position_grad.  Points must stay in the closed cell
 * (PIM_ERR_OUT_OF_CELL).  Synchronises.
 */
pim_status pim_update_positions(pim_plan plan, const double* xyz);

/*
 * pim_apply_batched -- u_i = A_i q_i (adjoint = 0) or A_i^H q_i (adjoint != 0)
 * for nplans plans -- several point sets, each with its own cell, grid and
 * kernel -- with nrhs right-hand sides each, as one unit of work.  The first
 * call with a given argument set (the plans, the q_i and u_i pointers, nrhs,
 * adjoint) is captured into a CUDA graph in which every plan's apply runs on
 * the plan's own stream, forked from and joined back to `stream`; identical
 * later calls replay that graph with a single launch.  Not part of the paper.
 *   plans, q, u  arrays of nplans entries; q[i], u[i] device pointers laid out
 *                as for pim_apply; a plan may appear only once.
 *   stream       cudaStream_t; NULL uses a library stream and synchronises.
 * The graphs of a plan are dropped by pim_set_points and pim_destroy (after
 * pim_update_positions a replay uses the new values, which are rewritten in
 * place).  Several right-hand sides (2..128) stream each plan's correction
 * list once for all of them.
 */
pim_status pim_apply_batched(int nplans, pim_plan const* plans, const void* const* q, void* const* u, int nrhs,
                             int adjoint, void* stream);

/*
 * pim_apply_noalloc -- pim_apply (adjoint = 0) or pim_apply_adjoint
 * (adjoint != 0) that allocates nothing: the per-call scratch of the apply
 * (sorted sources, box moments, the three grid work buffers, the far-zone
 * partial sums and far grids) comes from one 32 MiB device array that the
 * library holds on every GPU that loads it, until the process exits.  The
 * paper has no counterpart; this is for callers that cannot allocate device
 * memory when they apply the operator (a solver loop under a fixed memory
 * budget, code that runs while another thread captures a graph or owns the
 * stream-ordered allocator, bindings that can only pass in buffers they
 * already hold).  The plan itself is created beforehand as usual.
 *   q, u     device pointers only ([N][nrhs], as for pim_apply); host
 *            pointers -> PIM_ERR_ARG.
 *   Limit    plans whose scratch exceeds 32 MiB -> PIM_ERR_ARG with the
 *            required size in pim_last_error().
 *   Set-up   the first call on a device looks up the array's device address
 *            (cudaGetSymbolAddress) with that device current; make that first
 *            call before any stream capture.  The address is cached per device
 *            and per CUDA context: after the context is destroyed and created
 *            again (cudaDeviceReset) the next call looks it up again, so that
 *            call, too, belongs before any capture.
 *   Sharing  every call on a device uses the same array, which keeps the last
 *            call's contents (the apply writes every scratch word before it
 *            reads it, so nothing needs clearing); calls whose device work
 *            overlaps -- on different streams or from different threads --
 *            race.  Order them on one stream.  Calls on one plan from two
 *            threads at once also corrupt the plan itself (a call points the
 *            plan's scratch at the array for its duration): a plan is not
 *            thread safe.
 */
pim_status pim_apply_noalloc(pim_plan plan, const void* q, void* u, int nrhs, int adjoint, void* stream);

/* Device-side status of the calls issued so far: synchronises the plan's
 * streams, returns the first flag raised (PIM_OK if none) and clears it. */
pim_status pim_last_device_status(pim_plan plan);

/* Sizes and timings of a plan. */
pim_status pim_plan_info(pim_plan plan, pim_info* info);

/*
 * pim_set_profiling -- on != 0: every later apply records a CUDA event pair
 * around each pim_stage on the stream that stage runs on (a ring of 512
 * applies); on = 0 stops recording.  Either way the accumulated times are
 * cleared.  Events cost a few microseconds of device time per apply.
 */
pim_status pim_set_profiling(pim_plan plan, int on);

/*
 * pim_stage_times -- synchronises, then writes for each stage s < n the
 * total device time in ms (ms[s]) and the number of applies timed (count,
 * may be NULL) since pim_set_profiling.  Applies beyond the ring's 512 are
 * not included.
 */
pim_status pim_stage_times(pim_plan plan, double* ms, int n, int64_t* count);

/* Name of a stage ("spread", "fft", ...), static string; NULL if out of range. */
const char* pim_stage_name(int stage);

/*
 * pim_debug_copy -- copies an internal table to host memory, for tests of
 * individual stages.  `what`:
 *   0 far table G_far(delta o Delta + Delta/2), (2nf_x-1)(2nf_y-1)(2nf_z-1)
 *     complex128, x fastest;
 *   1 grid charges Q of the last apply (step 1), n_x n_y n_z, x fastest,
 *     complex of the plan precision (the last right-hand side);
 *   2 grid potential U of the last apply (step 2), same layout;
 *   3 sort permutation (int32, sorted slot -> caller index), N entries;
 *   4 correction row pointers (int64, N+1) in sorted order;
 *   5 correction columns (uint32, nnz): sorted column | image index << 25;
 *   6 correction values (complex128 FP64, nnz): G0 - G_grid before the phase;
 *   7 entries at the head of each row summed in double-float (int32, N;
 *     PIM_CORR_COMPACT plans only, PIM_ERR_STATE otherwise).
 * `bytes` must be at least the size of the table; PIM_ERR_ARG otherwise.
 */
pim_status pim_debug_copy(pim_plan plan, int what, void* host_out, size_t bytes);

/* Frees every resource of the plan (NULL is ignored). */
void pim_destroy(pim_plan plan);

#ifdef __cplusplus
}
#endif

#endif /* PIM_H */
