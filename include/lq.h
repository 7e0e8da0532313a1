/*
 * lq.h -- C ABI of the GB300 Wilson-Dirac library (liblq.so).
 *
 * The library applies the Wilson-Dirac operator of arXiv 1904.08616, Eq. (1),
 *
 *   (D psi)(n) = (m_q + 4) psi(n)
 *              + 1/2 sum_{mu=0..3} [ U_mu(n) P^{-mu} psi(n + mu) + U_mu(n - mu)^dag P^{+mu} psi(n - mu) ],
 *
 * its adjoint, and solves D^dag D x = eta by conjugate gradients, including the
 * residual-guided mixed-precision CG of the paper's Algorithm 1.  Every step runs in the
 * library's own CUDA kernels on one GPU (sm_103a).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * Lattice: dims[4] = {Lx, Ly, Lz, Lt}; every extent must be even and >= 2, and the volume
 *   V = Lx*Ly*Lz*Lt must satisfy V <= 10^8 (the largest volume the paper considers), and
 *   V * nrhs <= 2^28 (268,435,456) for calls on several fields.  Boundaries are periodic in all four
 *   directions.  Direction mu = 0, 1, 2, 3 is x, y, z, t.
 * Gamma matrices: chiral Euclidean basis, P^{-mu} = 1 - gamma_{mu+1}, P^{+mu} = 1 + gamma_{mu+1},
 *   gamma_k = [[0, -i sigma_k], [i sigma_k, 0]] (k = 1, 2, 3), gamma_4 = [[0, 1], [1, 0]],
 *   gamma_5 = diag(1, 1, -1, -1).  The hopping term carries the paper's "+1/2".
 * Site order, LQ_LAYOUT_LEX: n = x + Lx*(y + Ly*(z + Lz*t)), x fastest; site-major:
 *   spinor  [n][spin 4][colour 3][re, im]
 *   gauge   [n][mu 4][row r][col 3][re, im], r = 3 rows (LQ_LINK18) or the first 2 rows
 *           (LQ_LINK12; row 2 is rebuilt as conj(row0 x row1), exact for SU(3));
 *           LQ_LINK10: [n][mu 4][entry 5][re, im] = row 0 (u00, u01, u02), then the two
 *           entries of row 1 outside column k, in increasing column order.  k is the column
 *           of row 0 whose larger component max(|Re u0k|, |Im u0k|) is the largest (the lowest
 *           such column on ties), decided on the stored values.  Rebuilt: row 1's entry k from
 *           the orthogonality of rows 0 and 1, u1k = -(sum_{j != k} u1j conj(u0j)) / conj(u0k)
 *           (|u0k| >= 1/sqrt(6), so the division amplifies rounding by at most ~2.5), then
 *           row 2 as for LQ_LINK12; exact for SU(3) up to rounding.  The paper streams links
 *           as 10 words instead of 18 without trigonometric functions (Introduction,
 *           Section 2.2); its construction is not given, and this one is the library's.
 * Site order, LQ_LAYOUT_EO (parity-split structure of arrays, the fast internal layout):
 *   parity p = (x+y+z+t) mod 2, checkerboard index cb = n / 2, Vh = V / 2.  A field is cut
 *   into fixed-width chunks per site; chunk k of site (p, cb) is stored at chunk slot
 *     spinor:  (p*K + k)*Vh + cb
 *     gauge :  ((mu*2 + p)*K + k)*Vh + cb
 *   chunk widths in reals: spinor F64 2, F32 4, F16S 8, I32S 4; gauge LINK18 and LINK10 2
 *   (all precisions), LINK12 F64 2, F32 4, F16S 4, I32S 4; K = reals per site (24) or per
 *   link (18/12/10) / width.
 * Precisions (element types of the stored fields):
 *   LQ_F64  double; LQ_F32 float;
 *   LQ_F16S spinors: per site s = max |fl32(v)| over its 24 reals (float) and 24 halves
 *           h = fl16(fl32(v) / s) (h = 0 if s = 0); the buffer holds all halves first
 *           (48 V bytes, in the layout's order) followed by the V float scales (for EO the
 *           scale of (p, cb) is at p*Vh + cb).  The stored value is h * s.
 *           gauge fields: plain halves fl16(fl32(v)), no scale (SU(3) entries are <= 1).
 *   LQ_F64X FP64-class values as float pairs: hi = fl32(v), lo = fl32(v - hi), stored as the
 *           LQ_F64 field with every double replaced by (hi, lo) (same size and slots).
 *           Arithmetic: FP32-pair ("double-float") arithmetic, about 2^-47 relative, run on
 *           the FP32 pipes (GB300 executes FP64 at 1/63 of its FP32 rate).  LINK18 only.
 *   LQ_I32S 32-bit fixed point (Q1.30), the paper's FPGA-friendly format (Section 2.2):
 *           spinors: per site s = max |fl32(v)| over its 24 reals (float) and 24 int32
 *           q = RN(v / s * 2^30) (computed in FP64, ties to even; q = 0 if s = 0); all
 *           integers first (96 V bytes, in the layout's order), then the V float scales
 *           (EO: scale of (p, cb) at p*Vh + cb).  The stored value is q * s * 2^-30.
 *           gauge fields: int32 q = RN(u * 2^30) with no scale (entries must satisfy
 *           |u| < 2, as unitary links do).
 *   Arithmetic is FP64 for LQ_F64, FP32 pairs for LQ_F64X, FP32 for LQ_F32 / LQ_F16S /
 *   LQ_I32S (for LQ_F16S the operator forms each spin projection, one add of two stored
 *   values, in FP16 on the stored half2 words; every product and every sum of products is
 *   FP32).
 *   Kernel outputs in LQ_F16S use one reciprocal of the scale per site (h = fl16(v * fl32(1/s)));
 *   lq_convert_spinor divides every component (h = fl16(fl32(v) / s)) and is bit-exact.
 *   Kernel outputs in LQ_I32S use q = RN(fl32(v) * fl32(2^30 / s)) in FP32; lq_convert_spinor
 *   uses the FP64 definition above and is bit-exact.
 *
 * Several fields (right-hand sides) at once, nrhs of them:
 *   LEX: nrhs complete fields one after the other (field r at byte offset r * field size).
 *   EO : interleaved per site: chunk k of (p, cb) of field r at chunk slot
 *        ((p*K + k)*Vh + cb)*nrhs + r (F16S / I32S: all elements, then the scale of
 *        (p, cb, r) at (p*Vh + cb)*nrhs + r); for nrhs = 1 this is the single-field EO
 *        layout.  LEX stacks complete fields (F16S / I32S: each field's elements, then its
 *        scales).  The
 *        fields of one site sit side by side, so a batched kernel reads each link once for
 *        all of them.  EO multi-field buffers hold a power of two (<= 32) of fields.
 *
 * Buffers are device pointers owned by the caller, 16-byte aligned; the library neither
 * keeps nor frees them.  Calls that take a cuda_stream (a cudaStream_t, NULL = legacy
 * default stream) enqueue their kernels on it and return without waiting, except
 * lq_cg_solve, which returns after the solve has finished.
 *
 * Errors: every call returns an lq_status.  Arguments are checked before any kernel is
 * launched; on error nothing is written and lq_last_error() returns a message (per host
 * thread).  No call aborts, traps or throws across the ABI.
 */
#ifndef LQ_H
#define LQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum lq_status {
    LQ_OK = 0,
    LQ_NOT_CONVERGED = 1,     /* solver stopped at max_iter, max_cycles or stagnation (5 cycles
                                 without a new best true residual); x holds the last iterate   */
    LQ_ERR_ARG = -1,          /* bad enum value, null pointer, bad tolerance or count       */
    LQ_ERR_DIMS = -2,         /* odd, non-positive or too large lattice extents             */
    LQ_ERR_ALIGN = -3,        /* pointer not 16-byte aligned, or output aliases an input    */
    LQ_ERR_CUDA = -4,         /* a CUDA runtime call failed (message has the CUDA error)    */
    LQ_ERR_WORKSPACE = -5,    /* workspace missing or smaller than lq_cg_workspace_bytes()  */
    LQ_ERR_NONFINITE = -6,    /* a residual or a CG coefficient became NaN / Inf            */
    LQ_ERR_BREAKDOWN = -7     /* <p, D^dag D p> <= 0: the operator or the inputs are broken */
} lq_status;

typedef enum lq_prec { LQ_F64 = 0, LQ_F32 = 1, LQ_F16S = 2, LQ_F64X = 3, LQ_I32S = 4 } lq_prec;
typedef enum lq_link_fmt { LQ_LINK18 = 18, LQ_LINK12 = 12, LQ_LINK10 = 10 } lq_link_fmt;
typedef enum lq_layout { LQ_LAYOUT_LEX = 0, LQ_LAYOUT_EO = 1 } lq_layout;

/* Field kinds for lq_field_bytes. */
typedef enum lq_field_kind { LQ_FIELD_SPINOR = 0, LQ_FIELD_GAUGE = 1 } lq_field_kind;

/* Size in bytes of a stored field (spinor: link_fmt ignored). Returns 0 on bad arguments. */
size_t lq_field_bytes(const int32_t dims[4], int32_t kind, int32_t prec, int32_t link_fmt,
                      int32_t layout);

/*
 * lq_dslash_apply -- out = D psi, Eq. (1) of the paper (Introduction), on the whole lattice.
 *   m_q      quark mass of Eq. (1).
 *   prec     precision of U, psi and out (all three the same).
 *   link_fmt LQ_LINK18, LQ_LINK12 or LQ_LINK10 (12- and 10-real links are rebuilt in
 *            registers; LQ_F64X fields take LQ_LINK18 only).
 *   layout   LQ_LAYOUT_LEX or LQ_LAYOUT_EO, shared by U, psi and out.
 *   U, psi   inputs (device); out output (device), must not overlap psi or U.
 * One kernel launch on cuda_stream; returns without waiting.
 */
int lq_dslash_apply(const int32_t dims[4], double m_q, int32_t prec, int32_t link_fmt,
                    int32_t layout, const void *U, const void *psi, void *out,
                    void *cuda_stream);

/*
 * lq_dslash_adjoint -- out = D^dag psi.  The paper uses D^dag only inside D^dag D
 * (Algorithm 1, its three operator lines); it is Eq. (1) with P^{-mu} and P^{+mu}
 * exchanged, equal to gamma_5 D gamma_5.  Arguments as lq_dslash_apply.
 */
int lq_dslash_adjoint(const int32_t dims[4], double m_q, int32_t prec, int32_t link_fmt,
                      int32_t layout, const void *U, const void *psi, void *out,
                      void *cuda_stream);

/*
 * lq_dslash_apply_multi / lq_dslash_adjoint_multi -- out_r = D psi_r (or D^dag psi_r) for
 * nrhs fields at once, in the multi-field layouts above; the gauge field is read once per
 * site for all of them.  The paper applies D to one vector at a time (Eq. 1); batching is
 * this library's.  EO: nrhs a power of two <= 32, one launch.  LEX: any nrhs >= 1.
 */
int lq_dslash_apply_multi(const int32_t dims[4], double m_q, int32_t prec, int32_t link_fmt,
                          int32_t layout, int32_t nrhs, const void *U, const void *psi, void *out,
                          void *cuda_stream);
int lq_dslash_adjoint_multi(const int32_t dims[4], double m_q, int32_t prec, int32_t link_fmt,
                            int32_t layout, int32_t nrhs, const void *U, const void *psi, void *out,
                            void *cuda_stream);

/*
 * lq_dslash_hop -- the parity-to-parity hopping term of Eq. (1):
 *   out_p = a * y_p + b * H_{p,1-p} psi_{1-p},   H = 1/2 sum_mu [ ... ] of Eq. (1),
 * on the half lattice of parity out_parity (the even-odd split of Eq. 1; the paper does
 * not use it, it is this library's fast layout).  LQ_LAYOUT_EO only.  psi_other, y and out
 * are half fields: Vh sites of one parity, chunk slot k*Vh + cb (F16S / I32S: elements then the Vh
 * scales).  y may be NULL (then a is ignored); y may equal out.  dagger != 0 uses the
 * hopping term of D^dag.  One kernel launch.
 */
int lq_dslash_hop(const int32_t dims[4], int32_t out_parity, int32_t dagger, double a,
                  double b, int32_t prec, int32_t link_fmt, const void *U,
                  const void *psi_other, const void *y, void *out, void *cuda_stream);

/*
 * lq_convert_spinor / lq_convert_gauge -- re-encode a field into another precision,
 * link format or layout (the "pack/convert" step; the paper prepares its reduced link
 * form beforehand, Section 2.2).  Gauge sources must be LQ_LINK18; LQ_LINK12 keeps rows
 * 0 and 1, LQ_LINK10 row 0 and two entries of row 1 (column choice made on the rounded
 * row 0, as the header comment defines).  Rounding is round-to-nearest-even, through FP32 for FP16 targets; F16S
 * spinor encoding follows the rule in the header comment.  dst must not overlap src.
 */
int lq_convert_spinor(const int32_t dims[4], int32_t src_prec, int32_t src_layout,
                      const void *src, int32_t dst_prec, int32_t dst_layout, void *dst,
                      void *cuda_stream);
/* lq_convert_spinor for nrhs fields in the multi-field layouts (e.g. nrhs stacked FP64 LEX
 * fields into one interleaved FP32 EO buffer). */
int lq_convert_spinor_multi(const int32_t dims[4], int32_t nrhs, int32_t src_prec,
                            int32_t src_layout, const void *src, int32_t dst_prec,
                            int32_t dst_layout, void *dst, void *cuda_stream);
int lq_convert_gauge(const int32_t dims[4], int32_t src_prec, int32_t src_layout,
                     const void *src, int32_t dst_prec, int32_t dst_fmt, int32_t dst_layout,
                     void *dst, void *cuda_stream);

/* ---------------------------------------------------------------------------------- */
/* Conjugate gradient on D^dag D.                                                       */
/* ---------------------------------------------------------------------------------- */
typedef enum lq_cg_mode {
    LQ_CG_F64 = 0,        /* FP64 throughout (plain CG, true residual checked in FP64)     */
    LQ_CG_MIXED_F32 = 1,  /* Algorithm 1: FP32 inner loop (EO layout, 12-real links), FP64 outer */
    LQ_CG_MIXED_F16 = 2,  /* Algorithm 1: scaled-FP16 inner storage (the inner solution psi in
                             FP32), FP32 accumulation, FP64 outer                           */
    LQ_CG_F64X = 3,       /* FP64-class CG in FP32-pair arithmetic throughout (LQ_F64X)     */
    LQ_CG_MIXED_I32 = 4   /* Algorithm 1: 32-bit fixed-point inner storage (LQ_I32S), FP32
                             arithmetic, FP64 outer (not offered for lattice batches)      */
} lq_cg_mode;

typedef struct lq_cg_params {
    double tol;              /* stop when ||eta - D^dag D x|| <= tol ||eta|| (FP64)        */
    int32_t max_iter;        /* cap on inner iterations summed over all cycles (>= 1)      */
    int32_t max_cycles;      /* cap on outer cycles (reliable updates); 0 -> 1000          */
    double delta;            /* inner-loop residual reduction per cycle; <= 0 -> mode default
                                (MIXED_F32 / MIXED_I32 1e-4, MIXED_F16 1e-2, others 0)      */
    int32_t chunk;           /* host-driven inner loop: iterations between host checks;
                                0 -> automatic                                             */
    int32_t flags;           /* LQ_CG_PROFILE: time the solver's kernels with CUDA events  */
    int32_t max_inner;       /* cap on inner iterations per cycle (Algorithm 1's k); 0 -> 1000 */
} lq_cg_params;

/* lq_cg_params.flags */
#define LQ_CG_PROFILE 1      /* time the solver's kernels with CUDA events (see lq_cg_info)  */
#define LQ_CG_NATIVE_F64 2   /* outer residual and solution in native FP64 arithmetic instead
                                of FP32 pairs (mixed modes; slower on GB300)              */
#define LQ_CG_LINK18 4       /* inner links stored 18-real (no reconstruction) in the mixed
                                modes; default 12-real                                     */
#define LQ_CG_LINK10 32      /* inner links stored in the 10-real form (lq_cg_solve,
                                lq_cg_solve_multi and lq_cg_solve_noalloc in the mixed modes
                                with the FP32-pair outer loop; not with LQ_CG_LINK18 or
                                LQ_CG_NATIVE_F64)                                          */
#define LQ_CG_AUTOTUNE 8     /* lq_cg_solve_lattices: pick the inner block size by timing
                                (cached per lattice set and GPU); default 128 threads.
                                lq_cg_solve_multi without an LQ_CG_RHS_BLOCK_* flag: pick the
                                right-hand sides per thread (1, 2 or 4) by timing the two
                                inner stencil kernels on each batch of 2 or more (cached per
                                GPU, modes, lattice and batch size); default 1             */
#define LQ_CG_NO_GRAPH 16    /* drive the cycles from the host and launch the inner kernels
                                one by one, instead of running the whole solve's cycles in
                                one CUDA graph with conditional WHILE nodes (the default; if
                                the driver refuses such a graph the host-driven loop runs
                                without this flag too)                                     */
#define LQ_CG_RHS_BLOCK_1 0x1000 /* lq_cg_solve_multi: right-hand sides per thread in the inner
                                    stencil kernels (register blocking: each link is decoded once
                                    and applied to that many right-hand sides of a site); at most
                                    one flag, capped at the batch size; default 1 (blocking
                                    applies to mixed modes with 12-real inner links; the
                                    others always use 1)                                      */
#define LQ_CG_RHS_BLOCK_2 0x2000
#define LQ_CG_RHS_BLOCK_4 0x4000
#define LQ_CG_LATTICE_OWN_CYCLES 0x800 /* lq_cg_solve_lattices: each lattice takes its reliable
                                    update as soon as its own inner loop stops while the others
                                    go on (the host drives the cycles); by default every
                                    lattice's cycle ends together and the whole solve runs
                                    on the device as one graph launch                          */
#define LQ_CG_BLOCK_64 0x100 /* lq_cg_solve_lattices: inner block size 64 / 128 / 256 threads */
#define LQ_CG_BLOCK_128 0x200 /*   (at most one; overrides LQ_CG_AUTOTUNE)                  */
#define LQ_CG_BLOCK_256 0x400

/* Kernel roles reported in lq_cg_info.kernel_ms / kernel_calls. */
enum {
    LQ_K_APPLY_D = 0,        /* inner t = D p with ||t||^2                                  */
    LQ_K_APPLY_DDAG = 1,     /* inner q = D^dag t fused with the psi / r updates and ||r||^2 */
    LQ_K_UPDATE_P = 2,       /* inner p = r + beta p                                        */
    LQ_K_HIGH = 3            /* FP64 residual eta - D^dag D x (two operator kernels; four in
                                the Schur solve)                                           */
};

typedef struct lq_cg_info {
    int32_t status;          /* same value as returned                                     */
    int32_t iters;           /* inner iterations, all cycles                               */
    int32_t cycles;          /* outer cycles of Algorithm 1                                */
    int32_t high_applies;    /* applications of the FP64 D^dag D (Algorithm 1's residuals);
                                the first is skipped when the starting guess is zero      */
    double true_rel_resid;   /* ||eta - D^dag D x|| / ||eta||, FP64 operator, at return    */
    double eta_norm;         /* ||eta||                                                    */
    int32_t launches;        /* kernels this call launched (all roles, including skips)     */
    int32_t block;           /* threads per block of the inner stencil kernels               */
    double kernel_ms[4];     /* LQ_CG_PROFILE: summed device time per role (events)         */
    int32_t kernel_calls[4]; /* LQ_CG_PROFILE: launches that did work, per role             */
    int32_t rhs_block;       /* right-hand sides per thread of the inner stencil kernels     */
} lq_cg_info;

/* Workspace bytes lq_cg_solve needs for these dims and mode (0 on bad arguments). */
size_t lq_cg_workspace_bytes(const int32_t dims[4], int32_t mode);
/* Workspace bytes lq_cg_solve_multi needs for nrhs right-hand sides. */
size_t lq_cg_workspace_bytes_multi(const int32_t dims[4], int32_t mode, int32_t nrhs);

/*
 * lq_cg_solve -- solve D^dag D x = eta (Algorithm 1 of the paper, Section 1).
 *   U        gauge field, LQ_F64, LQ_LINK18, LQ_LAYOUT_LEX (device).
 *   eta      right-hand side, LQ_F64 LEX spinor (device).
 *   x        in: starting guess psi_0^high (Algorithm 1); out: solution (device,
 *            LQ_F64 LEX spinor; must not overlap eta, U or the workspace).
 *            The outer FP64-class quantities (psi^high, r^high, the residual operator) are held
 *            and computed as FP32 pairs (LQ_F64X) unless LQ_CG_NATIVE_F64 is set; LQ_CG_F64
 *            always uses native FP64.
 *   params   tolerances and caps (see lq_cg_params); NULL -> tol 1e-10, max_iter 100000.
 *            With LQ_CG_PROFILE set, CUDA events bracket the solver's kernels on cuda_stream
 *            and info reports their device time per role (inner launches that found the
 *            loop already stopped are not counted).
 *   workspace, ws_bytes  device scratch of at least lq_cg_workspace_bytes(dims, mode),
 *            16-byte aligned; its contents on entry are ignored.
 *   info     optional (host) statistics.
 * Kernels run on cuda_stream; the call returns after the solve has finished.  After the
 * set-up (field conversions, norms, the first outer residual) every cycle of Algorithm 1 runs
 * on the device as one CUDA graph launch: a conditional WHILE node over the cycles, each
 * holding the restart, a nested WHILE node over the inner iterations and the reliable update,
 * with every decision (convergence, limits, stagnation, the restart's parameters) taken by
 * one-thread kernels on the solver's state record; the host reads the record back once, at
 * the end.  With LQ_CG_PROFILE or LQ_CG_NO_GRAPH the host drives the cycles, launches the
 * inner kernels itself and polls the record between chunks of iterations.
 * Returns LQ_OK when the FP64 true residual meets tol, LQ_NOT_CONVERGED otherwise.
 */
int lq_cg_solve(const int32_t dims[4], double m_q, int32_t mode, const void *U,
                const void *eta, void *x, const lq_cg_params *params, void *workspace,
                size_t ws_bytes, lq_cg_info *info, void *cuda_stream);

/*
 * lq_cg_solve_noalloc -- lq_cg_solve without a caller workspace.  The paper has no
 * counterpart; this entry point exists for callers that cannot allocate device memory at
 * solve time: code under a no-allocation rule after start-up (real-time or reviewed
 * loops), plugins inside a host program whose allocator owns all device memory, or callers
 * with no CUDA allocator at hand.  They pass U, eta and x exactly as for lq_cg_solve; the
 * scratch is a fixed array inside this library (lq_cg_noalloc_max_workspace_bytes() bytes,
 * 64 MiB), which every GPU that loads the library holds until the process exits.
 *   - Lattices whose lq_cg_workspace_bytes(dims, mode) exceeds that size are rejected with
 *     LQ_ERR_WORKSPACE (12^4 fits in every mode, 16^4 in none).
 *   - The first call on a device looks up the array's device address (once per device,
 *     with that device current).  With CUDA's lazy module loading (the default) that first
 *     call is also when the array's memory is reserved on the device, so it can fail with
 *     LQ_ERR_CUDA for lack of memory: callers under a no-allocation rule make one call (a
 *     tiny solve) at start-up, before any stream capture.
 *   - The looked-up address is kept for the life of the process; resetting the device
 *     (cudaDeviceReset) while the library is loaded is not supported.
 *   - All calls share the one array, which keeps the previous call's contents; the solver
 *     re-initialises everything it reads.  Calls that overlap on the GPU (other streams,
 *     other host threads) race on the array and must not be issued.
 *   - Nothing is allocated: no cudaMalloc / cudaFree or allocating library routine.
 */
int lq_cg_solve_noalloc(const int32_t dims[4], double m_q, int32_t mode, const void *U,
                        const void *eta, void *x, const lq_cg_params *params, lq_cg_info *info,
                        void *cuda_stream);
size_t lq_cg_noalloc_max_workspace_bytes(void);

/*
 * lq_cg_solve_multi -- nrhs independent solves D^dag D x_r = eta_r (Algorithm 1 for each)
 * sharing the gauge field.  eta and x hold nrhs stacked FP64 LEX fields; info (optional)
 * receives nrhs records.  The right-hand sides are processed in batches of a power of two
 * (<= 8) whose kernels read each link once per site for the whole batch; each right-hand
 * side keeps its own CG scalars and stops on its own criterion while the batch goes on,
 * and the reliable updates of a batch are taken together.  Batching is not in the paper.
 * The mixed modes with 12-real inner links may serve several right-hand sides per thread
 * (LQ_CG_RHS_BLOCK_2/4), or choose that number per batch by timing (LQ_CG_AUTOTUNE; the
 * choice is cached per GPU, modes, lattice and batch size, and appended to the file named by
 * the environment variable LQ_TUNE_CACHE if set); info[r].rhs_block reports it.
 * Returns LQ_OK if every solve converged, LQ_NOT_CONVERGED if some did not, or the most
 * negative error status.
 */
int lq_cg_solve_multi(const int32_t dims[4], double m_q, int32_t mode, int32_t nrhs,
                      const void *U, const void *eta, void *x, const lq_cg_params *params,
                      void *workspace, size_t ws_bytes, lq_cg_info *info, void *cuda_stream);

/*
 * lq_cg_solve_schur -- solves D x_r = b_r (not D^dag D) for nrhs right-hand sides with the
 * even-odd Schur complement (not in the paper, which inverts D^dag D; the even-odd split of
 * Eq. 1 is this library's): with A = m_q + 4 and H the hopping term of Eq. (1),
 *   Mhat = A - H_eo H_oe / A on the even sites,  bhat_e = b_e - H_eo b_o / A,
 *   Mhat^dag Mhat x_e = Mhat^dag bhat_e by CG (Algorithm 1 in the mixed modes),
 *   x_o = (b_o - H_oe x_e) / A.
 * Every operator application is two half-lattice hops, the vectors are half fields, and
 * Mhat^dag Mhat is better conditioned than D^dag D.
 *   mode     LQ_CG_F64X, LQ_CG_MIXED_F32, LQ_CG_MIXED_F16 or LQ_CG_MIXED_I32 (the outer loop
 *            runs in FP32 pairs; LQ_CG_F64 and LQ_CG_NATIVE_F64 are rejected).
 *   b, x     nrhs stacked FP64 LEX fields; x holds the starting guess (its even half is used)
 *            and receives the solution.
 *   tol      relative to the normal equations: stop when
 *            ||Mhat^dag (bhat - Mhat x_e)|| <= tol ||Mhat^dag bhat||; info->true_rel_resid
 *            reports that ratio.
 *   workspace at least lq_cg_workspace_bytes_schur(dims, mode, nrhs) bytes.
 * Other arguments and the return value as lq_cg_solve_multi.
 */
size_t lq_cg_workspace_bytes_schur(const int32_t dims[4], int32_t mode, int32_t nrhs);
int lq_cg_solve_schur(const int32_t dims[4], double m_q, int32_t mode, int32_t nrhs,
                      const void *U, const void *b, void *x, const lq_cg_params *params,
                      void *workspace, size_t ws_bytes, lq_cg_info *info, void *cuda_stream);

/*
 * lq_cg_solve_lattices -- several independent problems, on lattices of different sizes,
 * solved together: for each lattice l, D_l^dag D_l x_{l,r} = eta_{l,r} for its nrhs
 * right-hand sides (Algorithm 1, or plain CG in LQ_CG_F64, per right-hand side as in
 * lq_cg_solve_multi).  Batching uneven lattices is not in the paper.
 *   n        number of lattices, 1 <= n <= 8.
 *   lats     n descriptors: dims, nrhs (1, 2, 4 or 8), m_q, and the caller's FP64 LEX
 *            fields U (18-real), eta and x (nrhs stacked fields each; x is the starting
 *            guess and receives the solutions).  No x may overlap another descriptor's
 *            fields or the workspace.
 *   mode     any lq_cg_mode; the mixed modes use 12-real inner links and FP32-pair outer
 *            arithmetic (LQ_CG_NATIVE_F64, LQ_CG_LINK18 and LQ_CG_PROFILE are rejected).
 *   params   as lq_cg_solve, plus LQ_CG_AUTOTUNE (choose the inner block size from 64, 128,
 *            256 by timing the first inner kernel over these lattices; the choice is cached
 *            per GPU, mode and lattice set, and appended to the file named by the
 *            environment variable LQ_TUNE_CACHE if set), LQ_CG_BLOCK_64/128/256 (a fixed
 *            inner block size) and LQ_CG_NO_GRAPH.
 *   workspace at least lq_cg_workspace_bytes_lattices(n, lats, mode) bytes.
 *   info     optional, sum of nrhs records in lattice order (block = the inner block size).
 * Each lattice's kernels use the grids a solve of that lattice alone would use, so every
 * lattice gets the result of its own solve, bit for bit.  By default the whole batch runs as
 * one CUDA graph launch: rounds of cycles in a conditional WHILE node, each round restarting
 * every lattice that needs a cycle, iterating all of them (each lattice's kernels a parallel
 * branch of the graph, running side by side) until every inner loop has stopped, and taking
 * each moved lattice's reliable update (Algorithm 1's outer step) under a conditional IF
 * node; all decisions are taken on the device.  Host-driven cycles issue the lattices'
 * kernels one lattice after the other.  With LQ_CG_LATTICE_OWN_CYCLES the host takes each
 * lattice's reliable update as soon as its own inner loop stops while the others go on.
 * Returns LQ_OK if every solve converged, LQ_NOT_CONVERGED if some did not, or the most
 * negative error status.  Returns after the solves have finished.
 */
typedef struct lq_lattice {
    int32_t dims[4];
    int32_t nrhs;
    int32_t pad;            /* set to 0 */
    double m_q;
    const void *U;
    const void *eta;
    void *x;
} lq_lattice;

size_t lq_cg_workspace_bytes_lattices(int32_t n, const lq_lattice *lats, int32_t mode);
int lq_cg_solve_lattices(int32_t n, const lq_lattice *lats, int32_t mode,
                         const lq_cg_params *params, void *workspace, size_t ws_bytes,
                         lq_cg_info *info, void *cuda_stream);

/*
 * Domain decomposition in t (the paper's multi-FPGA layout exchanges boundary data over
 * transceivers; Section 3): a lattice is cut into t-slabs, one per domain (rank), each
 * holding its own FP64 LEX 18-real links and spinors with local dims {Lx, Ly, Lz, Lt_local}
 * (Lx, Ly, Lz even >= 2, Lt_local >= 1).  Applying D on a domain needs two faces from its
 * neighbours in t, each Lx*Ly*Lz half spinors of 6 complex FP64 numbers
 * (lq_halo_face_bytes bytes):
 *   lq_halo_pack fills, from this domain's psi (and links),
 *     to_prev = (1 + S gamma_4) psi at t = 0, upper spin half (h0, h1), S = -1 for D and +1
 *               for D^dag: what the previous domain's forward t-hop needs;
 *     to_next = U_t^dag (1 - S gamma_4) psi at t = Lt_local - 1, upper half: what the next
 *               domain's backward t-hop needs (its link lives here).
 *     Face site s = x + Lx*(y + Ly*z).
 *   The caller delivers to_prev of domain r+1 as from_next of domain r and to_next of domain
 *   r-1 as from_prev of domain r (periodic in r).
 *   lq_halo_dslash then writes out = D psi (or D^dag psi, the same dagger as the pack) on the
 *   domain.  The result equals the single-domain lq_dslash_apply bit for bit.
 * Faces must not overlap out; one launch each.
 */
size_t lq_halo_face_bytes(const int32_t dims_local[4]);
int lq_halo_pack(const int32_t dims_local[4], int32_t dagger, const void *U, const void *psi,
                 void *to_prev, void *to_next, void *cuda_stream);
int lq_halo_dslash(const int32_t dims_local[4], double m_q, int32_t dagger, const void *U,
                   const void *psi, const void *from_next, const void *from_prev, void *out,
                   void *cuda_stream);

/*
 * lq_link_grad -- the gradient of L = Re <g, D psi> with respect to the links of Eq. (1),
 * for differentiating through the operator (the paper does not; this is the library's
 * adjoint support).  With the convention grad = dL/dRe U + i dL/dIm U, per link
 *   G_mu(n) = 1/2 sum_spin [ g(n) ((1 - gamma_mu) psi(n+mu))^H + ((1 + gamma_mu) psi(n)) g(n+mu)^H ],
 * a 3x3 complex matrix (colour row index from the first factor).  Differentiating through
 * D^dag uses lq_link_grad(psi, g) with the roles swapped, since Re <g, D^dag psi> =
 * Re <psi, D g>.  The mass term does not depend on U, so m_q is not an argument.
 *   g, psi : FP64 LEX spinor fields (V x 12 complex128), read only; the gradient is linear
 *            in each.
 *   out    : FP64 LEX 18-real gauge layout (V x 4 x 3 x 3 complex128), written as
 *            out = scale * G, or out += scale * G when accumulate != 0.  out must not
 *            overlap g or psi.
 * One kernel launch, asynchronous on cuda_stream; errors as for the other entry points.
 */
int lq_link_grad(const int32_t dims[4], const void *g, const void *psi, double scale,
                 int32_t accumulate, void *out, void *cuda_stream);

/*
 * lq_bounds_violations -- in the bounds-checked debug build (liblq_checked.so, compiled with
 * LQ_BOUNDS_CHECK; the stand-in for a memory checker), every field access of the operator and
 * solver kernels is checked against the slots of its field; an access out of range is skipped
 * (a load yields zero) and counted.  Returns the number of such accesses since the last call
 * (after waiting for the device) and, if any, the first offending slot index in *first
 * (optional); resets the count.  The normal build returns -1.  The paper has no counterpart.
 */
long long lq_bounds_violations(unsigned long long *first);

/* Message of the last error on this host thread ("" if none). */
const char *lq_last_error(void);

/* Library version string. */
const char *lq_version(void);

/* Short aliases with the operation names of the design (same semantics). */
int dslash_apply(const int32_t dims[4], double m_q, int32_t prec, int32_t link_fmt,
                 int32_t layout, const void *U, const void *psi, void *out, void *cuda_stream);
int dslash_adjoint(const int32_t dims[4], double m_q, int32_t prec, int32_t link_fmt,
                   int32_t layout, const void *U, const void *psi, void *out, void *cuda_stream);
int cg_solve(const int32_t dims[4], double m_q, int32_t mode, const void *U, const void *eta,
             void *x, const lq_cg_params *params, void *workspace, size_t ws_bytes,
             lq_cg_info *info, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* LQ_H */
