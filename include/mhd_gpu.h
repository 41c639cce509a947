/*
 * mhd_gpu.h -- C ABI of the GB300 (sm_103a) ghost-celled ideal-MHD patch
 * library: the hyperbolic advance of grid patches and the level operations
 * that feed it (ghost fill, prolongation/restriction, flux-register
 * refluxing, CFL time step, conservation sums).
 *
 * Method.  The AMR life cycle is that of Carroll-Nellenback et al.,
 * "Efficient Parallelization for AMR MHD Multiphysics Calculations" (Sec. 2.2:
 * Overlap, Prolongation, Advance, Synchronisation, Restriction).  Each patch
 * is advanced independently (Abstract, Sec. 2.3) with extended ghost zones of
 * width R * n_ghost (Sec. 2.3), updating a box that shrinks by n_ghost per
 * substep (Sec. 4, worked 4x4 example).  The paper does not state the MHD
 * solver; the advance is the unsplit MUSCL-Hancock scheme with primitive PLM
 * reconstruction, the HLLD Riemann solver of Miyoshi & Kusano (2005) and
 * constrained transport with Gardiner & Stone (2005) upwinded edge EMFs.  One
 * step consumes n_ghost = 2 ghost layers.
 *
 * Memory.  The caller owns every state array and every stream; the library
 * owns its context, its scratch arena and its device copies of descriptor
 * and copy lists.  State is structure-of-arrays: five cell arrays (rho, Mx,
 * My, Mz, E) and three face arrays (Bx on x-faces, By on y-faces, Bz on
 * z-faces) that share one set of element strides (stride[0] == 1, x fastest).
 * A patch with interior box [lo, hi] and g ghost layers has N_d = hi_d - lo_d
 * + 1 + 2g cells per axis; array index a_d = global index - (lo_d - g); face
 * arrays carry one extra entry (index N_d) along their normal, and face index
 * a is the lower face of cell a.  Every array must hold at least
 * stride[2] * (N_2 + 1) elements.  Elements are double (MHD_F64) or float
 * (MHD_F32); flux registers and conservation sums are always double.
 *
 * Execution.  Every call that takes a stream enqueues work on it and returns
 * without synchronising, except mhd_get_device_status and mhd_ctx_destroy.
 * Arguments that can be checked on the host are checked before anything is
 * launched; a failed check returns a negative status and launches nothing.
 * Errors found on the device (a non-positive density or pressure after an
 * update) set a status word read by mhd_get_device_status; kernels never trap.
 * A context may be used from one host thread at a time.  All calls of a
 * context share its scratch arena: calls on different streams must be ordered
 * by the caller (events), or use one context per stream.  Device tables are
 * cached by content, so after one warm-up call with the same arguments a call
 * uploads nothing and can be captured in a CUDA graph; a captured graph holds
 * the scratch address, which changes only when a larger call grows the arena.
 */
#ifndef MHD_GPU_H
#define MHD_GPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t mhd_status;
#define MHD_OK 0
#define MHD_EINVAL (-1)    /* bad argument (host check)                      */
#define MHD_ENOMEM (-2)    /* the library could not allocate its scratch     */
#define MHD_ECUDA (-3)     /* a CUDA runtime call failed                     */
#define MHD_ENEGATIVE (-4) /* device: rho <= 0 or p <= 0 after an update      */
#define MHD_ETIMEOUT (-5)  /* device: a bounded wait gave up                  */
#define MHD_ETOOBIG (-6)   /* request exceeds a fixed static capacity        */

#define MHD_F64 0
#define MHD_F32 1

typedef struct mhd_ctx mhd_ctx;

/* Inclusive box of cells in a level's global index space. */
typedef struct {
  int32_t lo[3], hi[3];
} mhd_box;

/* One patch (grid, Sec. 2): its interior box on its level, its ghost width
 * and its arrays.  Pointers are device pointers to elements of `dtype`. */
typedef struct {
  int32_t level;     /* refinement level l (dx_l = dx_0 / R^l, Sec. 2)        */
  int32_t nghost;    /* g: ghost layers on every side                       */
  int32_t dtype;     /* MHD_F64 or MHD_F32                                  */
  int32_t patch_id;  /* caller's id, echoed in error messages               */
  mhd_box interior;  /* cells owned by the patch                            */
  void *U[5];        /* rho, Mx, My, Mz, E                                  */
  void *B[3];        /* Bx, By, Bz                                          */
  int64_t stride[3]; /* element strides; stride[0] must be 1                */
  double dx[3];      /* cell widths                                         */
} mhd_patch_desc;

/* Solver constants.  The paper fixes none of them. */
typedef struct {
  double gamma;      /* ratio of specific heats, > 1                        */
  double cfl;        /* Courant number, in (0, 1]                           */
  int32_t limiter;   /* 0 van Leer harmonic, 1 minmod, 2 monotonised central */
  int32_t emf;       /* 0 Gardiner-Stone upwinded, 1 arithmetic mean        */
  double upwind_eps; /* contact speeds |S_M| <= upwind_eps (S_R - S_L) count as
                        no upwind side in the EMF upwinding; <= 0 selects
                        1e-10 for MHD_F64 and 1e-5 for MHD_F32 patches      */
  int32_t fp64_contract; /* MHD_F64 advance: 0 the parity build (no fused
                        multiply-add; every operation rounded as written, in
                        the oracle's order), 1 the build with multiply-adds
                        fused (about 1.25x faster; differs from 0 by rounding) */
  int32_t advance_kernel; /* 0: the context's choice (the staged kernels until
                        mhd_autotune_advance measured something else faster);
                        1: the staged kernels (one launch per stage,
                        intermediates in the scratch arena; the predictor
                        tiled in shared memory if the autotuner chose it);
                        2: the fused kernel (one persistent launch over x-y
                        tiles marching along z, intermediates in shared
                        memory); 3: the staged kernels with the predictor
                        tiled in shared memory; 4: the fused pass (one
                        kernel for the primitives, the predictor and the
                        Riemann fluxes over x-y tiles marching along z, the
                        predicted face states kept on chip), then the staged
                        EMF and update kernels.  All compute every element
                        with the same expressions; a call whose captures need
                        face fluxes outside the update box runs staged (2) or
                        takes them from the fused pass's flux planes (4).   */
  int32_t fused_chunk; /* z-planes per work item of the fused kernel (2) or
                        of the fused pass (4); 0 lets each call choose (from
                        the device's SM count for 2, 16 planes for 4)        */
  int32_t kernel_shape; /* compiled tile shape of the fused kernel (2) or of
                        the fused pass (4): 0 the context's choice (the first
                        shape until mhd_autotune_advance chose one); s >= 1
                        shape s - 1 of the element type's table: fused pass
                        FP32 1: 16 x 16, 2: 16 x 12, 3: 24 x 8, 4: 16 x 8
                        cells, FP64 1: 8 x 8; fused kernel FP32 1-4: 16 x 16
                        (512 threads), 16 x 16, 16 x 12, 24 x 8 (384), FP64
                        1: 8 x 8.  A shape outside the table of a call's
                        element type is MHD_EINVAL at that call.            */
  double p_floor;    /* floors, applied after every update to the cells of
                        the update box (and by mhd_floor): a density below
                        rho_floor becomes rho_floor with M kept and the
                        pressure reset to p_floor; otherwise a pressure (from
                        the new face field) below p_floor gets E raised by
                        (p_floor - p) / (gamma - 1).  Not conservative; the
                        changed cells are counted (mhd_floor_count).  0: no
                        floor (the paper names none).                       */
  double rho_floor;  /* see p_floor; 0: no density floor                    */
} mhd_params;

/* One ghost-fill copy (Sec. 2.2, the step that refreshes ghost cells from
 * neighbours; Sec. 2.3): `box` (global index space of the destination's level) is an
 * image of src's interior (source index = destination index + `offset`, a
 * periodic shift or zero) clipped to dst's ghost-extended box grown by one
 * cell.  Every box cell that lies in dst's arrays takes src's values, and so
 * does every face of a box cell that exists in dst's face arrays (the outer
 * cell layer supplies the faces on the outer planes of those arrays), except
 * faces of dst's interior (normal index in [lo, hi+1], other indices inside
 * the interior).  A face that is the upper face of one box's top layer and
 * the lower face of another box's bottom layer takes the first box's value
 * (both sources hold that face); with that rule the copies of one call write
 * disjoint elements, and a call is one launch.  The boxes of one destination
 * must not overlap (their cells would be written twice, in no fixed order),
 * source boxes must lie in src's interior, and copies of one call must read
 * only interiors.  A box may hold at most 2^24 - 1 rows (y-z extent
 * product); a larger one returns MHD_EINVAL. */
typedef struct {
  int32_t src, dst;    /* indices into the descriptor array                 */
  mhd_box box;         /* destination cells                                 */
  int32_t offset[3];   /* source global index = destination index + offset  */
} mhd_copy;

/* AMR items (refinement ratio 2; fine global index = 2 x coarse + {0, 1};
 * fine patches are aligned: even lower corner, even extent). */
typedef struct {
  int32_t coarse, fine; /* indices into the coarse / fine descriptor arrays  */
  mhd_box box;          /* coarse cells, coarse global index                 */
} mhd_prolong_item;

typedef struct {
  int32_t fine, coarse;
  mhd_box box;          /* coarse cells: the coarsened fine interior clipped
                           to the coarse interior grown by one cell          */
} mhd_restrict_item;

#define MHD_CAP_FACE 0
#define MHD_CAP_EDGE 1

/* Flux-register capture of an advance (FP64): kind MHD_CAP_FACE stores
 * dt * F (rho, Mx, My, Mz, E: 5 planes over the box, x fastest) on the
 * axis-normal faces of `box` (face index = index of the cell above the
 * face); MHD_CAP_EDGE stores dt * E_axis (1 plane) on the axis edges of `box`
 * (an edge is indexed by the cell at whose lower corner lines it lies).
 * mode 0 writes, 1 adds (accumulation over substeps).  box: global index of
 * the patch's level; it must lie within the faces / edges the advance
 * computes (faces: normal index in [lo-k, hi+k+1], others in
 * [lo-k-1, hi+k+1]; edges: along axis [lo-k, hi+k], others [lo-k, hi+k+1]). */
typedef struct {
  int32_t patch, kind, axis, mode;
  mhd_box box;
  double *dst;          /* device                                            */
} mhd_capture;

#define MHD_REFLUX 0
#define MHD_SYNC 1

/* One flux-register deposit (Sec. 2.2: restriction of fluxes from the fine
 * level and synchronisation of fluxes).
 * mode MHD_REFLUX (coarse-fine faces): for each coarse face of `box` (kind
 * MHD_CAP_FACE, normal `axis`) the correction
 *   dF_q = 0.25 * (sum of the 4 fine sub-face registers) - coarse register,
 * for each coarse edge (kind MHD_CAP_EDGE, along `axis`)
 *   dE = 0.5 * (sum of the 2 fine segment registers) - coarse register;
 * fine: register over fine_box (fine global index, x fastest); coarse_reg:
 * register over box.
 * mode MHD_SYNC (faces or edges shared by two patches of one level, whose two
 * registers differ when the patches computed them from different data): the
 * patch `coarse` is corrected to the mean of the two registers,
 *   dF_q = 0.5 * (other - own),  dE = 0.5 * (other - own),
 * with `coarse_reg` its own register over box and `fine` the other patch's
 * register over fine_box, which must equal box (one level, one index
 * space); give one deposit per patch of the pair.  Where the two registers
 * agree (R14: the usual case after a ghost fill from identical data) the
 * correction is exactly zero and nothing changes.
 * Either way the correction goes into the patch's correction planes (18
 * FP64 planes with the patch's strides: plane 5 d + q holds dF_q of axis-d
 * faces, plane 15 + a the axis-a dE). */
typedef struct {
  int32_t coarse, kind, axis, mode;   /* mode: MHD_REFLUX or MHD_SYNC         */
  mhd_box box;          /* global index of the corrected patch's level       */
  mhd_box fine_box;
  const double *fine;   /* device                                            */
  const double *coarse_reg;
} mhd_deposit;

/* Context: owns scratch memory and device copies of small host tables on
 * CUDA device `device`.  *out is NULL on failure. */
mhd_status mhd_ctx_create(const mhd_params *params, int32_t device, mhd_ctx **out);
/* A new context on the device of src with src's parameters and advance
 * choices (those the autotuner stored included), and its own scratch arena,
 * tables, status word and timer: the way to run calls of one solver
 * configuration concurrently on several streams (each stream its own
 * context), as the level-concurrent AMR step does (Sec. 4).  *out is NULL on
 * failure; MHD_EINVAL for NULL arguments. */
mhd_status mhd_ctx_clone(const mhd_ctx *src, mhd_ctx **out);
void mhd_ctx_destroy(mhd_ctx *ctx);
const char *mhd_last_error(const mhd_ctx *ctx);

/* CFL time step (Sec. 2.2 advances with dt_l = dt_{l-1}/R): writes to the
 * device double *d_dt_out the minimum over patches p and interior cells of
 *   scale[p] * cfl * min_d dx_d / (|v_d| + c_f,d),
 * c_f,d the fast magnetosonic speed along d (Bc = mean of the two faces).
 * scale (host, length n, may be NULL for all ones) is R^level for the
 * coarse-step dt of a hierarchy.  The minimum is exact (order independent). */
mhd_status mhd_cfl_dt(mhd_ctx *ctx, const mhd_patch_desc *patches, int32_t n,
                      const double *scale, double *d_dt_out, void *stream);

/* Advance (A of Sec. 2.2) of n patches by one step of dt_p = (*d_dt) *
 * dt_scale[p] (d_dt a device double, dt_scale host, may be NULL for ones).
 * Patch p updates its interior grown by grow[p] layers (host array, may be
 * NULL for zeros) and the face fields on that box; it needs valid data on
 * the interior grown by grow[p] + 2 and requires grow[p] + 2 <= nghost
 * (Sec. 2.3: the update box shrinks by n_ghost = 2 per substep).  Patches
 * must not share memory.  caps (host, ncap entries, may be NULL) capture
 * dt * F and dt * E of this step into FP64 flux registers (mhd_capture).  On
 * return the work is enqueued on `stream`. */
mhd_status mhd_patch_advance(mhd_ctx *ctx, const mhd_patch_desc *patches, int32_t n,
                             const int32_t *grow, const double *d_dt,
                             const double *dt_scale, const mhd_capture *caps,
                             int32_t ncap, void *stream);

/* One single-level step whose dt is the CFL time step of the state it starts
 * from: writes to the device double *d_dt_out what mhd_cfl_dt (scale NULL)
 * would, then advances the n patches (update box = interior, no captures) by
 * that dt as mhd_patch_advance does.  The staged kernels compute the CFL
 * reduction inside the primitive pass (the same expressions, so the same dt
 * in the FP64 parity build), which saves reading the state a second time;
 * the fused kernel runs the separate reduction first.  For a hierarchy, whose
 * dt is a minimum over all levels (Sec. 2.2), use mhd_cfl_dt and
 * mhd_patch_advance.  Errors as mhd_patch_advance. */
mhd_status mhd_patch_step_cfl(mhd_ctx *ctx, const mhd_patch_desc *patches, int32_t n, double *d_dt_out,
                              void *stream);

/* Autotuner of the advance (no counterpart in the paper; it picks how the
 * patches of a call are advanced).  Times, on these patches (update box grown
 * by grow[p], may be NULL for zeros; dt from *d_dt), every compiled tile
 * shape of the fused pass (advance_kernel 4), the staged kernels with the
 * untiled and with the shared-memory-tiled predictor, and every compiled tile
 * shape of the fused kernel of the patches' element type, the fused pass and
 * the fused kernel each with a few z-chunk lengths: reps launches after one
 * warm-up, with the new state written to the context's scratch only, so the
 * patch state is unchanged, and with a status word of their own, so that the
 * context's device status is unchanged too.  caps / ncap (may be NULL / 0) are the flux-
 * register captures the real calls make, as for mhd_patch_advance: they are
 * not written, but the candidates do the extra stores that feed them, and the
 * fused kernel is left out when a real call could not run it.  The fastest becomes this context's advance for
 * that element type (mhd_params.advance_kernel = 0; mhd_params.fused_chunk > 0
 * still fixes the chunk).  Synchronises `stream`.  Outputs (may be NULL): the
 * choice (-3 - s: the fused pass of advance_kernel 4 in shape s of its table;
 * -2 staged with the untiled predictor, the default before tuning; -1 staged
 * with the tiled one; s >= 0 the fused kernel in shape s), the chunk length (0
 * for staged) and the time per advance in milliseconds. */
mhd_status mhd_autotune_advance(mhd_ctx *ctx, const mhd_patch_desc *patches, int32_t n,
                                const int32_t *grow, const mhd_capture *caps, int32_t ncap,
                                const double *d_dt, int32_t reps,
                                int32_t *choice_out, int32_t *chunk_out, float *ms_out,
                                void *stream);

/* Prolongation (P of Sec. 2.2: pre-advance coarse data into the fine ghost
 * zones, Sec. 2.3) of the coarse cells of each item into its fine patch: the
 * 8 fine cells get U_c + (+-h_x) + (+-h_y) + (+-h_z), h_d = 0.25 minmod of the
 * coarse one-sided differences (conservative limited linear); the faces of
 * those fine cells (lower faces, plus the array's extra upper face) get a
 * divergence-free reconstruction inside the coarse cell (Balsara 2001 for
 * R = 2): each coarse face contributes its value and its minmod transverse
 * quarter-slopes, and the quadratic field matching those traces with
 * div B = 0 gives the inner faces.  The fine patch's own interior faces are
 * never written.  The coarse cells and their one-cell stencil must lie in the
 * coarse arrays, the fine cells in the fine arrays.  Coarse and fine patches
 * share one dtype. */
mhd_status mhd_prolong(mhd_ctx *ctx, const mhd_patch_desc *coarse, int32_t nc,
                       const mhd_patch_desc *fine, int32_t nf,
                       const mhd_prolong_item *items, int32_t n, void *stream);

/* Restriction (R of Sec. 2.2): every item cell inside the coarse interior =
 * 0.125 (sum of its 8 fine cells); every face of an item cell that is a face
 * of the coarse interior = 0.25 (sum of its 4 fine sub-faces).  Lower faces
 * are written in a first pass and upper faces in a second, so a coarse face
 * covered by two fine patches, or owned by two coarse patches, gets one
 * value. */
mhd_status mhd_restrict(mhd_ctx *ctx, const mhd_patch_desc *fine, int32_t nf,
                        const mhd_patch_desc *coarse, int32_t nc,
                        const mhd_restrict_item *items, int32_t n, void *stream);

#define MHD_PROLONG 0
#define MHD_RESTRICT 1

/* One coarse-fine item of mhd_restrict_prolong: `box` holds coarse cells
 * (coarse global index) under the rules of mhd_prolong (mode MHD_PROLONG) or
 * mhd_restrict (mode MHD_RESTRICT). */
typedef struct {
  int32_t fine, coarse; /* indices into the fine / coarse descriptor arrays  */
  mhd_box box;
} mhd_level_item;

/* The P and R operations of Sec. 2.2 behind one entry point: mode
 * MHD_PROLONG runs mhd_prolong (coarse -> fine ghost zones), MHD_RESTRICT
 * runs mhd_restrict (fine -> covered coarse cells and faces), with the same
 * checks, results and errors; any other mode is MHD_EINVAL. */
mhd_status mhd_restrict_prolong(mhd_ctx *ctx, int32_t mode, const mhd_patch_desc *fine,
                                int32_t nf, const mhd_patch_desc *coarse, int32_t nc,
                                const mhd_level_item *items, int32_t n, void *stream);

/* Refluxing (Sec. 2.2: fine fluxes restricted to the coarse level at the
 * coarse-fine boundary): executes the deposits into the correction planes
 * corr[p] (host array of nc device pointers, NULL for coarse patches without
 * children; 18 FP64 planes each, see mhd_deposit), then corrects every
 * interior cell and face of those coarse patches:
 *   U_q -= (dF_x(+x) - dF_x)/dx - (dF_y(+y) - dF_y)/dy - (dF_z(+z) - dF_z)/dz,
 *   B_a -= (dE_c(+b) - dE_c)/dx_b - (dE_b(+c) - dE_b)/dx_c   (b, c = a+1, a+2),
 * in FP64 (FP32 state is rounded once).  The planes must be all zero on entry
 * (zero them once after allocation); the call zeroes the elements its
 * deposits wrote before returning, so they are zero again for the next call,
 * and it touches only the cells and faces next to deposited elements (all
 * others have a zero correction).  Call mhd_restrict afterwards: it
 * overwrites the covered cells and faces. */
mhd_status mhd_reflux(mhd_ctx *ctx, const mhd_patch_desc *coarse, int32_t nc,
                      double *const *corr, const mhd_deposit *deps, int32_t nd,
                      void *stream);

/* Library-owned FP64 flux registers (Sec. 2.2: the fluxes of a patch's
 * boundary kept for the synchronisation and refluxing steps).  For each of the
 * n patches (host array of descriptors; only the interiors are read) the
 * library allocates on the context's device
 *   - six boundary-face registers: side s of axis d covers the axis-d faces
 *     with normal index lo_d (s = 0) or hi_d + 1 (s = 1) and transverse
 *     indices over the interior: 5 planes (dt F of rho, Mx, My, Mz, E), x
 *     fastest, the layout of a face capture over that box;
 *   - twelve boundary-edge registers, two per boundary face: the axis-a
 *     edges (a one of the face's two transverse axes) that lie in side s of
 *     axis d, i.e. normal index lo_d (s = 0) or hi_d + 1 (s = 1), index
 *     lo_a .. hi_a along a and lo_t .. hi_t + 1 along the remaining axis t:
 *     1 plane (dt E_a), the layout of an edge capture over that box.
 * All are zero after creation.  mhd_fluxreg_face / mhd_fluxreg_edge return
 * the device pointer of one register (NULL for a bad index) and its box, to
 * be named as mhd_capture.dst and as mhd_deposit.fine / coarse_reg; the
 * library frees them in mhd_fluxreg_destroy (after synchronising the
 * device).  MHD_EINVAL for bad arguments, MHD_ENOMEM if the allocation
 * fails. */
typedef struct mhd_fluxreg mhd_fluxreg;
mhd_status mhd_fluxreg_create(mhd_ctx *ctx, const mhd_patch_desc *patches, int32_t n, mhd_fluxreg **out);
void mhd_fluxreg_destroy(mhd_fluxreg *reg);
double *mhd_fluxreg_face(const mhd_fluxreg *reg, int32_t patch, int32_t axis, int32_t side, mhd_box *box);
double *mhd_fluxreg_edge(const mhd_fluxreg *reg, int32_t patch, int32_t face_axis, int32_t side,
                         int32_t edge_axis, mhd_box *box);
/* Zeroes every register of `reg` on `stream` (asynchronous). */
mhd_status mhd_fluxreg_zero(mhd_fluxreg *reg, void *stream);

/* Ghost fill (Sec. 2.2 S step: ghost cells refreshed; periodic images and
 * same-level neighbours): executes the copies of `list` (host array) in one
 * launch.  All patches of the call must have one dtype. */
mhd_status mhd_ghost_fill(mhd_ctx *ctx, const mhd_patch_desc *patches, int32_t n,
                          const mhd_copy *list, int32_t nlist, void *stream);

/* Conservation sums over the interiors of n patches (one dtype):
 * d_out8[q] = sum of U_q dV (q < 5) and of B_{q-5} dV over the lower faces of
 * interior cells (q >= 5), accumulated in double in a fixed order (the result
 * is reproducible run to run).  d_out8 is a device array of 8 doubles. */
mhd_status mhd_conservation_sums(mhd_ctx *ctx, const mhd_patch_desc *patches, int32_t n,
                                 double *d_out8, void *stream);

/* The same conservation sums, for callers that cannot allocate memory (the
 * paper has no counterpart).  Some callers own no device memory of their own:
 * their process's memory is reserved by another allocator (a serving
 * framework's caching pool), or they must not call cudaMalloc/cudaFree because
 * those calls can synchronise the device and stall other streams, or they run
 * as a plugin that is not allowed to allocate.  This entry point needs no
 * context and allocates nothing, on the device or the host: the partial sums
 * live in a fixed array inside the library (1 MiB per GPU, held by every GPU
 * that loads the library until the process exits) and the descriptors travel
 * as a kernel argument.  The caller passes the patches (host array) and
 * d_out8 (device, 8 doubles), as for mhd_conservation_sums, and gets the same
 * values bit for bit; the work is enqueued on `stream` of the current device.
 * Limits: at most 16 patches and 4,194,304 interior cells in total (16384
 * blocks of 256 cells); larger requests return MHD_ETOOBIG and launch
 * nothing; bad descriptors return MHD_EINVAL.  The first call on each device
 * looks up the array's device address (cudaGetSymbolAddress with that device
 * current), and so does the first call after the device's context changed
 * (cudaDeviceReset); make such a first call before any stream capture.  All calls on a
 * device share the array: calls that overlap on the GPU (different streams
 * without ordering between them) race and may return wrong sums. */
mhd_status mhd_conservation_sums_static(const mhd_patch_desc *patches, int32_t n,
                                        double *d_out8, void *stream);

/* Synchronises the context's device, then returns (and clears) the device
 * status word in *out: MHD_OK or the first device error raised since the
 * last call.  The return value reports CUDA failures of the call itself. */
mhd_status mhd_get_device_status(mhd_ctx *ctx, int32_t *out);

/* Library version and build flags (for logs). */
const char *mhd_version(void);

/* ---- AMR tree on the device (Sec. 3.1: neighbour inheritance) ----------
 * Boxes are int32 device arrays lo[3 n], hi[3 n] (inclusive, level index
 * space, x first).  CSR offsets are int64 device arrays of length n + 1.
 * Both calls are pure functions of their device inputs (no context, nothing
 * allocated); each runs in two passes: with the output list NULL it writes
 * one count per element into d_count, with it non-NULL it writes the entries
 * of element i at positions d_off[i] ... (offsets from the counts).  They
 * enqueue one kernel on `stream` and return MHD_EINVAL for bad arguments
 * (nothing launched) or MHD_ECUDA if the launch fails. */

/* Parents of nf fine boxes (level l+1) among nc coarse boxes (level l): the
 * coarse boxes that meet the fine box coarsened by 2 ([floor(lo/2),
 * floor(hi/2)]), listed in increasing index order.  A fine box of a properly
 * nested hierarchy lies inside the union of its parents. */
mhd_status mhd_tree_parents(const int32_t *d_flo, const int32_t *d_fhi, int32_t nf, const int32_t *d_clo,
                            const int32_t *d_chi, int32_t nc, const int64_t *d_off, int32_t *d_count,
                            int32_t *d_list, void *stream);

/* Interactions of the n boxes of level l+1 inherited from level l (Sec. 3.1:
 * the neighbours of a node's children are children of the node's
 * neighbours).  For box c: every (c', s) such that c' is a child of P' (kid
 * CSR of level l, the transpose of the parents lists), (P', s) is an
 * interaction of a parent P of c (par CSR of the children; int CSR of level
 * l with shifts s in {-1, 0, 1}^3 as three int8 per entry), and box(c') + s
 * ndom meets box(c) grown by r cells (ndom: cells per side of the periodic
 * level-(l+1) domain).  Entries come in loop order (parents, their
 * interactions, their children) and may repeat; (c, 0) itself is included.
 * If the level-l interactions hold every pair at range r, the output holds
 * every such pair of level l+1 (nesting makes the inheritance complete).  A
 * virtual root (one parent of every level-0 box, interacting with itself
 * under all 27 shifts) gives the brute-force pairs of level 0. */
mhd_status mhd_tree_inherit(const int32_t *d_lo, const int32_t *d_hi, int32_t n, int32_t ndom, int32_t r,
                            const int64_t *d_par_off, const int32_t *d_par, const int64_t *d_int_off,
                            const int32_t *d_int, const int8_t *d_int_shift, const int64_t *d_kid_off,
                            const int32_t *d_kid, const int64_t *d_out_off, int32_t *d_count, int32_t *d_out,
                            int8_t *d_out_shift, void *stream);

/* ---- Space-filling-curve ordering and Hilbert splitting (Sec. 5.1, 5.2) ----
 * Hilbert index: Skilling's transposed-axes construction of the Hilbert
 * curve through [0, 2^bits)^dim (dim 2 or 3; bits <= 30 in 2-D, <= 20 in
 * 3-D).  The curve starts at the origin, steps between face neighbours, and
 * gives the 2^dim children of a cell (coordinates 2x .. 2x+1) one contiguous
 * block of indices, so that child order follows parent order (Sec. 5.1).
 * The distance of a grid along the curve is the sum of the indices of its
 * 2^dim corner cells (Sec. 5.1 samples a grid by its corners). */

/* Keys of n_pts points: d_pts int32 device array [n_pts][dim] (coordinates
 * of one point together), d_keys uint64 device array of n_pts; a point
 * outside [0, 2^bits)^dim gets the key UINT64_MAX.  Enqueues one kernel on
 * `stream`; MHD_EINVAL for bad arguments (nothing launched), MHD_ECUDA if the
 * launch fails. */
mhd_status mhd_hilbert_keys(const int32_t *d_pts, int64_t n_pts, int32_t dim, int32_t bits, uint64_t *d_keys,
                            void *stream);

/* Distances of n_boxes inclusive boxes (d_lo, d_hi int32 device arrays
 * [n_boxes][dim]) into d_dist (int64 device array); a box that is empty or
 * leaves [0, 2^bits)^dim gets INT64_MAX.  Same launch and errors as
 * mhd_hilbert_keys. */
mhd_status mhd_box_distances(const int32_t *d_lo, const int32_t *d_hi, int64_t n_boxes, int32_t dim,
                             int32_t bits, int64_t *d_dist, void *stream);

/* Hilbert splitting of the inclusive box [lo, hi] (host arrays of dim
 * values, inside [0, 2^bits)^dim) into one piece per weight (host array of
 * n_weights positive finite values), by the recursive bisection of Sec. 5.2:
 * the weight list is cut where the two sums differ least (ties to the
 * shorter prefix); each axis of extent >= 2 is cut next to the proportional
 * point (floor and ceiling), with the prefix's piece on the low or on the
 * high side; the candidate whose slower piece has the least cells-with-ghosts
 * (extent + 2 ghost per axis) per unit of weight wins, and among candidates
 * within 1% of that cost the one whose suffix piece leads the prefix piece
 * furthest along the curve; both pieces are split again with their weights.
 * Writes the pieces, in weight order, to the host arrays out_lo, out_hi
 * [n_weights][dim].  Host code only (no device work).  MHD_EINVAL for bad
 * arguments or when a piece of one cell would have to be split. */
mhd_status mhd_hilbert_split(const int32_t *lo, const int32_t *hi, int32_t dim, const double *weights,
                             int32_t n_weights, int32_t bits, int32_t ghost, int32_t *out_lo, int32_t *out_hi);

/* ---- Grid generation for regridding (Sec. 2.1) ----
 * Boxes covering the flagged cells of a level: the paper leaves the rule
 * open; this is the point clustering of Berger & Rigoutsos (IEEE Trans. SMC
 * 21, 1278 (1991)).  flags: host uint8 array of shape[0] x ... x shape[dim-1]
 * cells (dim 2 or 3, C order: the last index fastest), nonzero = flagged.  A
 * box is shrunk to its flags' bounding box and accepted when flagged cells /
 * cells >= eff (0 < eff <= 1) or when no axis is at least 2 min_size long;
 * otherwise it is cut, both pieces at least min_size long, at the signature
 * hole nearest its centre (axes in order), else at the largest sign change of
 * the signature's second difference, else at the middle of its longest axis,
 * and both pieces are clustered again (low piece first).  Writes the boxes
 * (inclusive, in the flag array's index space and axis order) to the host
 * arrays out_lo, out_hi [max_boxes][dim] and their number to *n_out.  Host
 * code only.  MHD_EINVAL for bad arguments; MHD_ETOOBIG (with *n_out set)
 * when more than max_boxes boxes result. */
mhd_status mhd_cluster_flags(const uint8_t *flags, int32_t dim, const int32_t *shape, double eff,
                             int32_t min_size, int32_t max_boxes, int32_t *out_lo, int32_t *out_hi,
                             int32_t *n_out);

/* Measured ALU peak of the current device (diagnostics for the roofline of
 * the advance; no counterpart in the paper): times, with CUDA events, one
 * launch of a kernel in which every thread of (SM count x 8) blocks of 256
 * threads runs 16 independent multiply-add chains for `iters` iterations, in
 * FP32 (dtype MHD_F32) or FP64 (MHD_F64), after one shorter warm-up launch.
 * Writes the rate in TFLOP/s (2 flops per multiply-add) to *tflops and the
 * timed launch's duration to *ms.  Synchronous: it allocates a small device
 * buffer, a stream and two events of its own, waits for the kernel and frees
 * them.  MHD_EINVAL for bad arguments, MHD_ECUDA if a CUDA call fails. */
mhd_status mhd_alu_probe(int32_t dtype, int32_t iters, double *tflops, double *ms);

/* Error flags for regridding (Sec. 2.1: each iteration of a level flags the
 * cells that need refinement; the paper leaves the criterion to the
 * application).  An interior cell is flagged when the normalised central
 * difference of the density or of the pressure along some axis exceeds theta:
 *   |q(+d) - q(-d)| > theta (|q(+d)| + 2 |q| + |q(-d)|),  q in {rho, p},
 * evaluated in FP64 (an FP32 state is converted first; p from the
 * cell-centred field, the mean of the two faces).  d_flags (device) receives
 * one byte per interior cell (1 flagged, 0 not), patch after patch, each
 * patch's interior x fastest.  Needs one valid ghost layer.  Asynchronous on
 * `stream`; MHD_EINVAL for bad arguments.  mhd_cluster_flags turns the flags
 * of a level into grids. */
mhd_status mhd_flag_cells(mhd_ctx *ctx, const mhd_patch_desc *patches, int32_t n, double theta,
                          uint8_t *d_flags, void *stream);

/* Data transfer into a new iteration of a level (regridding, Sec. 2.1: a
 * new grid takes the previous iteration's data where the two meet, and is
 * prolonged from the parent level elsewhere; the O step of Sec. 2.2).
 *
 * mhd_transfer_copy: for every item, copies from old patch `src` (index into
 * `old`) to new patch `dst` (index into `fresh`), both of one level and one
 * dtype: kind -1 the five cell arrays over the cells of `box`, kind a (0..2)
 * the axis-a face array over the faces of `box` (index along a = face index).
 * Give the cells of the intersection of the two interiors and, per axis, the
 * faces common to both patches' face sets (normal index in [lo, hi + 1] of
 * both, the others in both interiors), so that a new patch that only touches
 * an old one still takes the old value of the face they share.
 * MHD_EINVAL for an index or a box outside the arrays (nothing launched). */
typedef struct {
  int32_t src, dst, kind, pad;
  mhd_box box;          /* global index of the level                          */
} mhd_transfer_item;
mhd_status mhd_transfer_copy(mhd_ctx *ctx, const mhd_patch_desc *old, int32_t no, const mhd_patch_desc *fresh,
                             int32_t nn, const mhd_transfer_item *items, int32_t ni, void *stream);

/* mhd_prolong_new: prolongation of the coarse cells of each item's `box`
 * (coarse global index; coarse patch `coarse`, new fine patch `fine`) into
 * the fine patch's interior: the eight children and every face of them, the
 * fine patch's own boundary faces included.  Each coarse cell is governed by
 * its byte of the item's mask (device, one byte per coarse cell of
 * mask_box, x fastest):
 *   bit 0          the children already hold the previous iteration's data
 *                  (mhd_transfer_copy): nothing is written;
 *   bit 1 + 2a + s the four sub-faces on side s of axis a already hold the
 *                  previous iteration's values: they are kept and read.
 * Cells: density and momentum limited-linear (minmod quarter slopes, as
 * mhd_prolong); energy_mode 0: the thermal energy prolonged the same way
 * (as mhd_prolong), energy_mode 1: the children's thermal energies then
 * scaled by (1 + delta / ebar) so that their total energies average to the
 * coarse cell's (delta = E_c - mean child energy, ebar = mean child thermal
 * energy; left unscaled, and counted in *d_fallbacks (device, nullable), where
 * ebar + delta <= 0).  Faces: Balsara's divergence-free reconstruction (as
 * mhd_prolong) on the faces not kept; where a coarse cell keeps sub-faces, its
 * twelve inner fine faces are changed by the least-squares correction that
 * zeroes every child's divergence given the kept values (the gradient of the
 * cube-Laplacian potential of the children's divergences).  Equal cell
 * widths along the three axes; old patches aligned to the coarse grid.
 * MHD_EINVAL for bad indices or boxes (nothing launched). */
typedef struct {
  int32_t coarse, fine;
  mhd_box box;          /* coarse cells, coarse global index                  */
  const uint8_t *mask;  /* device                                             */
  mhd_box mask_box;     /* coarse global index, contains box                  */
} mhd_prolong_new_item;
mhd_status mhd_prolong_new(mhd_ctx *ctx, const mhd_patch_desc *coarse, int32_t nc, const mhd_patch_desc *fine,
                           int32_t nf, const mhd_prolong_new_item *items, int32_t ni, int32_t energy_mode,
                           unsigned long long *d_fallbacks, void *stream);

/* Synchronises the context's device, then returns in *out the number of
 * cells that the floors (mhd_params.p_floor, rho_floor) changed since the
 * last call, and resets the count. */
mhd_status mhd_floor_count(mhd_ctx *ctx, int64_t *out);

/* The context's floors (mhd_params.p_floor, rho_floor) applied to every
 * interior cell of the patches, e.g. after refluxing, which changes cells
 * outside any advance.  Asynchronous; nothing is launched when both floors are
 * 0.  MHD_EINVAL for bad arguments. */
mhd_status mhd_floor(mhd_ctx *ctx, const mhd_patch_desc *patches, int32_t n, void *stream);

/* Number of kernels this context has enqueued so far (for launch accounting). */
int64_t mhd_launch_count(const mhd_ctx *ctx);

/* Per-kernel event timer (diagnostics, no counterpart in the paper).  While
 * enabled, every launch of the context is bracketed by two CUDA events
 * recorded on the launching stream.  mhd_timing_read synchronises on the
 * pending events and returns, for kernel id `kernel` (0 <= id < 16, names from
 * mhd_kernel_name), the summed device time in ms and the number of launches
 * since the last reset; mhd_timing_reset clears the sums. */
mhd_status mhd_timing_enable(mhd_ctx *ctx, int32_t on);
mhd_status mhd_timing_read(mhd_ctx *ctx, int32_t kernel, double *total_ms, int64_t *launches);
mhd_status mhd_timing_reset(mhd_ctx *ctx);
const char *mhd_kernel_name(int32_t kernel);

#ifdef __cplusplus
}
#endif
#endif /* MHD_GPU_H */
