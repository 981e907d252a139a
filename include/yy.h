/*
 * yy.h - C ABI of the Yin-Yang multipole gravity solver (GB300, sm_103a).
 *
 * Computes the Newtonian potential Phi and the field -grad(Phi) of a
 * cell-averaged density given on the two patches of a Yin-Yang grid, by the
 * multipole method of Almanstotter, Melson, Janka & Mueller (2018),
 * "Parallelized solution method of the three-dimensional gravitational
 * potential on the Yin-Yang grid" (arXiv:1806.04593), which builds on
 * Mueller & Steinmetz (1995).
 *
 * Per solve, on the caller's CUDA stream and without host synchronisation:
 *   analysis   A_p[i][lm] = sum_jk rho_p[i][jk] w_jk K_lm T_j^(lm) {C_k^(m), S_k^(m)}
 *              (§3 Eqs. ac/as with the overlap weight of §4), both patches;
 *   radial     inner / outer sums of Eqs. phiin/phiout at the interfaces
 *              r_n^+, as scaled prefix / suffix scans over r;
 *   combine    the other patch's moments re-expressed in each patch's frame
 *              (a fixed rotation within each degree l) and added to its own,
 *              so that one set of coefficients per patch gives the §4 sum
 *              Phi(r_q) = Phi_q(r_q) + Phi_p(r_q) (the other patch's terms are
 *              its harmonics at the target points in its own angles,
 *              Eqs. trafotheta/trafophi);
 *   synthesis  Phi on both patches from the combined coefficients and the
 *              own-frame harmonics; optionally -grad(Phi) in the target
 *              patch's local spherical basis.
 *
 * Conventions (all functions):
 *  - Arrays are C-contiguous float64.  A patch field is [n_r][n_theta][n_phi]
 *    (radius slowest, phi fastest); a gradient is [3][n_r][n_theta][n_phi]
 *    holding (g_r, g_theta, g_phi).
 *  - Zone i (0-based) spans r_edges[i]..r_edges[i+1]; output row n is the
 *    outer interface r = r_edges[n+1] (the paper evaluates at interfaces).
 *    Density is zero inside r_edges[0].
 *  - Patch cells: theta_j = pi/4 - delta_theta + (j + 1/2) d_theta with
 *    d_theta = (pi/2 + 2 delta_theta)/n_theta, phi_k = -3pi/4 - delta_phi +
 *    (k + 1/2) d_phi with d_phi = (3pi/2 + 2 delta_phi)/n_phi (§4 intervals).
 *    Outputs are at the cell-centre angles of the target patch.
 *  - The Yang patch's local Cartesian frame is (x,y,z) -> (-x,z,y) of Yin's.
 *  - Device pointers must be 16-byte aligned.  Input and output buffers are
 *    owned by the caller; the handle owns its tables and workspace.
 *  - A handle is not thread-safe and must be used from one stream at a time.
 *  - Arguments are validated on the host; a failed check returns
 *    YY_ERR_INVALID_ARG before any device work.  The library never aborts,
 *    never uses device assert or trap, and never synchronises inside
 *    yy_potential.  Kernels that detect a bad condition set a device error
 *    word that yy_last_device_status reports.
 */
#ifndef YY_H
#define YY_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct yy_grid yy_grid;

typedef enum {
  YY_OK = 0,
  YY_ERR_INVALID_ARG = 1,
  YY_ERR_OOM = 2,
  YY_ERR_CUDA = 3,
  YY_ERR_NOT_SUPPORTED = 4,
  YY_ERR_TIMEOUT = 5,
  YY_ERR_DEVICE_CHECK = 6
} yy_status;

/* Arithmetic of the two contractions (analysis and synthesis).  Tables and
 * the radial scans are float64 in every form.
 *   YY_FP64   float64 operands and accumulation (CUDA-core DFMA).
 *   YY_FP32   float32 operands and accumulation (CUDA-core FFMA).
 *   YY_TF32   one tf32 product per term on tcgen05 tensor cores, fp32 accumulation.
 *   YY_BF16X3 operands split into 3 bf16 terms, 6 cross products, fp32
 *             accumulation per K chunk, chunks summed in float64.
 *   YY_FP16X2 operands split into 2 scaled fp16 terms, 3 cross products,
 *             fp32 accumulation per K chunk, chunks summed in float64.
 *   YY_FP64_OZAKI  float64 results (the YY_FP64 tolerance) with the
 *             azimuthal stages of the separable analysis and synthesis on
 *             tcgen05 tensor cores by the Ozaki scheme: the rows (rho w, the
 *             polar-stage sums G) and the azimuthal / trig tables written as
 *             six balanced 8-bit digits (integers exact in bf16) under a
 *             power-of-two scale per row, the 26 digit products of levels
 *             <= 6 accumulated exactly in fp32 per level, levels combined in
 *             integers and rounded once to float64.  The polar stages and
 *             the combination of the patches run in float-float arithmetic
 *             (unevaluated pairs of fp32 values, about 48 bits: exact
 *             products by fused multiply-add and exact sums by TwoSum) on the
 *             CUDA cores' fp32 pipe, each input scaled by a power of two that
 *             follows the data; the radial scans are float64 as for YY_FP64
 *             (and so is the analysis with YY_ANALYSIS_DENSE, or with more
 *             than 640 cells per row).  Multiplying rho by a power of two
 *             multiplies every result by the same power exactly.
 *             Needs yy_grid_prepare and 2 l_max + 1 <= 127 (l_max <= 63);
 *             above l_max 30 the contractions take their general kernels
 *             (no spare bias columns in G rows of 64 slots, rows of 128
 *             slots past l_max 31, the analysis in tiles of 32 slots). */
typedef enum {
  YY_FP64 = 0,
  YY_FP32 = 1,
  YY_TF32 = 2,
  YY_BF16X3 = 3,
  YY_FP16X2 = 4,
  YY_FP64_OZAKI = 5
} yy_precision;

/* Tables and intermediates readable through yy_grid_copy_table (tests and
 * diagnostics).  Mode index: idx(l,0) = l^2, idx(l,m,cos) = l^2 + 2m - 1,
 * idx(l,m,sin) = l^2 + 2m (m >= 1), n_lm = (l_max+1)^2.
 *   YY_TABLE_WEIGHTS  [n_theta][n_phi]       overlap weights w_jk (§4)
 *   YY_TABLE_TBAR     [n_theta][n_lm]        K_lm T_j^(lm) (Eq. tlm), cos and sin slots equal
 *   YY_TABLE_ANALYSIS [n_lm][n_theta*n_phi]  w_jk K_lm T_j^(lm) {C_k^(m), S_k^(m)}
 *   YY_TABLE_SYNTH    [n_theta*n_phi][n_lm]  K_lm P_l^m {cos, sin}(m phi) at the cell centre
 *   YY_TABLE_SYNTH_T  same layout: d/dtheta
 *   YY_TABLE_SYNTH_P  same layout: (1/sin theta) d/dphi
 *   YY_TABLE_MOMENTS  [2 n_r][n_lm]          normalised A of each patch's own cells in
 *                                            its own frame, last solve (Yin rows first)
 *   YY_TABLE_COEFF    [3][2 n_r][n_lm]       synthesis coefficients of the last solve:
 *                                            Phi, g_r, angular gradient
 *   YY_TABLE_ROTATION [sum_l (2l+1)^2]       per degree l, the (2l+1) x (2l+1) matrix D^l
 *                                            (row-major, at offset l (4l^2-1)/3) with
 *                                            Y_i(other-patch angles) = sum_j D^l_ij Y_j(own
 *                                            angles); modes of degree l in index order
 *   YY_TABLE_MOMENTS_TOTAL [2 n_r][n_lm]     moments of both patches in each patch's
 *                                            frame: A_p + D^T A_(other), last solve */
typedef enum {
  YY_TABLE_WEIGHTS = 0,
  YY_TABLE_TBAR = 1,
  YY_TABLE_ANALYSIS = 2,
  YY_TABLE_SYNTH = 3,
  YY_TABLE_SYNTH_T = 4,
  YY_TABLE_SYNTH_P = 5,
  YY_TABLE_MOMENTS = 6,
  YY_TABLE_COEFF = 7,
  YY_TABLE_ROTATION = 8,
  YY_TABLE_MOMENTS_TOTAL = 9
} yy_table;

/* How the analysis and the synthesis are evaluated (yy_grid_set_analysis).
 *   YY_ANALYSIS_AUTO (default)  separable analysis and synthesis for YY_FP64
 *       and YY_FP32; dense contractions for the tensor-core forms (there the
 *       tensor cores outrun the separable stages despite 12.6 times the
 *       flops).  Grids whose tables overflow the separable kernels' shared
 *       memory use the dense evaluation.
 *   YY_ANALYSIS_SEPARABLE  the weight folded into the density, then
 *       an azimuthal stage (cell integrals C_k^(m), S_k^(m)) and a polar stage
 *       (K_lm T_j^(lm)): 2 n_ang (2 l_max + 1) + 2 n_theta n_lm flops per shell.
 *       Float64 for YY_FP64; for the other forms fp32 on CUDA cores with the
 *       m = 0 sums (the monopole) carried in float64.
 *       The synthesis is separable too: a polar stage
 *       G[t] = sum_l q[l^2 + t] K_lm P_l^m (theta_j) and an azimuthal stage
 *       sum_t G[t] {cos, sin}(m phi_k); for the tensor-core forms the polar
 *       stage runs on CUDA cores and the azimuthal one on the tensor cores
 *       with G and the trig table as three bf16 pieces (the t = 0 term, which
 *       holds the monopole, added per cell).
 *   YY_ANALYSIS_DENSE  one contraction of the densities with the full
 *       analysis table, 2 n_ang n_lm flops per shell, in the form's arithmetic
 *       (tensor cores for YY_TF32 / YY_BF16X3 / YY_FP16X2), and the synthesis
 *       as dense contractions with the full harmonic tables.
 * All give the §3 moments A_p (Eqs. ac/as with the §4 weights) and the §2
 * sums of Eq. potential.                                                   */
typedef enum {
  YY_ANALYSIS_AUTO = 0,
  YY_ANALYSIS_SEPARABLE = 1,
  YY_ANALYSIS_DENSE = 2
} yy_analysis;

/* Create a grid handle on the current CUDA device and build every
 * density-independent term once (§3: the constant terms are computed only
 * while the grid is fixed): overlap weights, polar / azimuthal integrals,
 * normalised harmonic tables at the cell centres and their angular
 * derivatives, the per-degree rotation between the two patches' harmonics,
 * and the radial scan coefficients, all in float64 on the GPU.  Synchronises the device before returning.
 *   r_edges      host, n_r + 1 values, r_edges[0] >= 0, strictly increasing
 *   n_r          radial zones, 1 <= n_r <= 1<<20
 *   n_theta/phi  cells per patch, >= 1 each, n_theta * n_phi <= 1<<24
 *   delta_theta  buffer widths (radians), 0 <= delta < pi/4
 *   delta_phi
 *   l_max        0 <= l_max <= 80
 *   G            gravitational constant (finite)
 *   out          receives the handle (set to NULL on failure)
 * Errors: YY_ERR_INVALID_ARG, YY_ERR_OOM, YY_ERR_CUDA. */
yy_status yy_grid_create(const double *r_edges, int n_r, int n_theta, int n_phi,
                         double delta_theta, double delta_phi, int l_max, double G,
                         yy_grid **out);

/* Create a handle for the full spherical polar grid of §2 (the comparison
 * grid of §5): one patch, theta_j^+- = (j, j+1) pi / n_theta and
 * phi_k^+- = (k, k+1) 2 pi / n_phi in the global frame, every cell counted
 * once (w = 1), no second patch and no rotation table.  Arguments, rules and
 * errors as for yy_grid_create without the buffer widths.  For this handle
 * yy_potential and yy_potential_host take the Yin arguments only and require
 * rho_yang, phi_yang and grad_yang to be NULL; the per-patch tables hold n_r
 * rows instead of 2 n_r, and YY_TABLE_ROTATION gives YY_ERR_NOT_SUPPORTED. */
yy_status yy_polar_grid_create(const double *r_edges, int n_r, int n_theta, int n_phi, int l_max,
                               double G, yy_grid **out);

/* Select the analysis evaluation for later solves (see yy_analysis).
 * YY_ANALYSIS_SEPARABLE builds the separable tensor-core tables of every
 * tensor-core form already prepared (allocates device memory, synchronises;
 * a form prepared later while it is selected builds them in yy_grid_prepare).
 * They stay until the handle is destroyed or the batch tuner drops them for a
 * field that does not use them.  Must not be called while a stream is being
 * captured unless the tables already exist.
 * Errors: YY_ERR_INVALID_ARG; YY_ERR_OOM / YY_ERR_CUDA from building the
 * tables (the method stays selected; those forms then use the dense path). */
yy_status yy_grid_set_analysis(yy_grid *g, yy_analysis method);

/* K split of the dense analysis (YY_ANALYSIS_DENSE, or AUTO where it picks
 * the dense evaluation) for one form: the number of tiles along the K axis
 * (n_ang cells) that run side by side.  K is cut into segments fixed by the
 * grid's sizes; each segment's products are summed in one fixed order into a
 * partial of its own, a split takes whole segments, and the partials are
 * added in segment order.  So the moments A -- and everything computed from
 * them -- are bitwise the same for every split; the split changes only the
 * speed.  (Sec. 3, the paragraph on the global summation of A_C and A_S:
 * there the order of the sums changed with the number of tasks, and
 * double-double sums made A reproducible; here the order is fixed instead.)
 *   yy_grid_analysis_splits returns the current split (-1 for a NULL handle
 *   or an unknown form; 0 for a tensor-core form not prepared yet) and, when
 *   not NULL, writes the sizes' default to *rule and the largest accepted
 *   split (the number of segments) to *max_splits.  YY_FP64, YY_FP32 and
 *   YY_FP64_OZAKI (whose dense analysis is that of YY_FP64) share the
 *   CUDA-core contraction's split.
 *   yy_grid_set_analysis_splits sets it (0: the default) for later solves.
 *   Errors: YY_ERR_INVALID_ARG (NULL, unknown form, splits < 0 or above
 *   *max_splits); YY_ERR_NOT_SUPPORTED (tensor-core form not prepared). */
int yy_grid_analysis_splits(const yy_grid *g, yy_precision prec, int *rule, int *max_splits);
yy_status yy_grid_set_analysis_splits(yy_grid *g, yy_precision prec, int splits);

/* Build the operand tables of a reduced-precision form or of YY_FP64_OZAKI
 * (allocates device memory; synchronises).  YY_FP64 is always ready.
 * Returns YY_ERR_NOT_SUPPORTED if the device cannot run the form, or for
 * YY_FP64_OZAKI when l_max > 63. */
yy_status yy_grid_prepare(yy_grid *g, yy_precision prec);

/* One solve on `cuda_stream` (a cudaStream_t, NULL = legacy default stream).
 *   rho_yin, rho_yang   device, [n_r][n_theta][n_phi] float64 (read)
 *   phi_yin, phi_yang   device, same shape (written)
 *   grad_yin, grad_yang device, [3][n_r][n_theta][n_phi] or both NULL
 * On a polar grid (yy_polar_grid_create) the Yang pointers must be NULL.
 * Asynchronous; no host synchronisation.  Errors: YY_ERR_INVALID_ARG (NULL
 * or misaligned pointer, one gradient pointer NULL), YY_ERR_NOT_SUPPORTED
 * (precision not prepared), YY_ERR_CUDA (launch failure). */
yy_status yy_potential(yy_grid *g, const double *rho_yin, const double *rho_yang,
                       double *phi_yin, double *phi_yang,
                       double *grad_yin, double *grad_yang,
                       yy_precision prec, void *cuda_stream);

/* yy_potential with HOST buffers: copies rho to the handle's device staging
 * buffers, solves, copies Phi (and the gradient) back, and synchronises the
 * stream before returning.  Host buffers should be page-locked for full
 * copy bandwidth.  The first call allocates the staging buffers. */
yy_status yy_potential_host(yy_grid *g, const double *rho_yin, const double *rho_yang,
                            double *phi_yin, double *phi_yang,
                            double *grad_yin, double *grad_yang,
                            yy_precision prec, void *cuda_stream);

/* Pipelined form of yy_potential_host for a stream of solves: enqueues the
 * copy in, the solve (on cuda_stream) and the copy out, and returns without
 * waiting.  Two staging sets alternate between calls, and the copies run on
 * the handle's own streams, so the copy out of one call overlaps the copy in
 * and the solve of the next (host-device copies run at about 200 GB/s in each
 * direction on this machine; a solve with the gradient moves 1.07 GB).  The
 * host buffers of a call must stay valid and untouched until the results are
 * in: after yy_potential_host_wait, or two calls later for its input.  Use one
 * cuda_stream for all calls on a handle.  Errors as for yy_potential_host. */
yy_status yy_potential_host_async(yy_grid *g, const double *rho_yin, const double *rho_yang,
                                  double *phi_yin, double *phi_yang,
                                  double *grad_yin, double *grad_yang,
                                  yy_precision prec, void *cuda_stream);

/* Wait until every yy_potential_host_async call on the handle has delivered
 * its results to host memory. */
yy_status yy_potential_host_wait(yy_grid *g);

/* Copy a table or intermediate (see yy_table) into host memory; `count` is
 * the number of float64 values the caller's buffer holds and must equal the
 * table's size (query it with host_dst = NULL: *count receives the size).
 * Synchronises the device. */
yy_status yy_grid_copy_table(yy_grid *g, yy_table which, double *host_dst, size_t *count);

/* Device error word of the handle (synchronises the device).  YY_OK or
 * YY_ERR_DEVICE_CHECK / YY_ERR_TIMEOUT; reading clears it. */
yy_status yy_last_device_status(yy_grid *g);

/* Release the handle and all its device memory (NULL-safe; synchronises). */
void yy_destroy(yy_grid *g);

/* Static description of a status code. */
const char *yy_status_string(yy_status s);

/* Stage timing (diagnostics).  When enabled, yy_potential records CUDA
 * events on its stream at the stage boundaries; yy_grid_stage_ms synchronises
 * and returns the durations of the last solve in milliseconds:
 *   ms[YY_STAGE_ANALYSIS]   analysis contraction (operand packing included)
 *   ms[YY_STAGE_SCAN]       moment combination and radial scans (coefficient
 *                           packing included)
 *   ms[YY_STAGE_SYNTHESIS]  synthesis of Phi and, when requested, -grad Phi
 *                           (one or four contractions)                      */
typedef enum {
  YY_STAGE_ANALYSIS = 0,
  YY_STAGE_SCAN = 1,
  YY_STAGE_SYNTHESIS = 2,
  YY_STAGE_COUNT = 3
} yy_stage;
yy_status yy_grid_set_profiling(yy_grid *g, int enable);
yy_status yy_grid_stage_ms(yy_grid *g, double *ms);

/* Per-kernel timing (diagnostics).  While profiling is enabled, yy_potential
 * also records a CUDA event on its stream after each kernel it launches (the
 * first 32).  For the last solve, kernel `index` (0 <= index <
 * yy_last_launch_count) gets *ms = the time from the end of the kernel before
 * it (from the solve's start for index 0) to its own end, and *name = a static
 * string naming the kernel (not to be freed).  Synchronises on that event.
 * Errors: YY_ERR_INVALID_ARG (profiling off, index out of range). */
yy_status yy_grid_kernel_ms(yy_grid *g, int index, double *ms, const char **name);

/* Radial inner / outer sums without a handle and without any allocation.
 * (No counterpart in the paper: this is a deployment variant of the scan.)
 * For callers that cannot allocate device memory where they need the sums:
 * applications whose device memory is owned entirely by their own pool or
 * arena, hosts that load this code as a plugin and forbid it the allocator,
 * and time-critical loops where cudaMalloc / cudaFree (which may synchronise
 * the device) are not allowed.  It computes the same coefficients as the
 * solve's scan stage.
 *   r_edges  device, n_r + 1 radii obeying yy_grid_create's rules (not
 *            checked here; values that break them give undefined results)
 *   moments  device, [2 n_r][n_lm] normalised moments, Yin rows first: the
 *            combined moments of YY_TABLE_MOMENTS_TOTAL
 *   coeff    device out, [3][2 n_r][n_lm]: the Phi, g_r and angular-gradient
 *            coefficients, in the layout of YY_TABLE_COEFF
 *   n_r >= 1, 0 <= l_max <= 80, G finite; pointers 8-byte aligned (the
 *   kernel reads and writes single float64 values).
 * Scratch: a static device array of 2^21 float64 (16 MiB) that every GPU
 * loading the library keeps until exit; 2 n_r (l_max+1)^2 must not exceed
 * 2^21, otherwise YY_ERR_INVALID_ARG and nothing is launched.  Nothing in the
 * scratch needs clearing (each value is written before it is read), but all
 * calls share it: calls whose kernels overlap on the GPU (other streams,
 * other threads) race and give wrong results.  The first call on a device
 * (and again the first call after its context is recreated, for example by
 * cudaDeviceReset) does the set-up: it looks up the array's device address
 * (cudaGetSymbolAddress), which allocates nothing; make that first call
 * before any stream capture.  Asynchronous on cuda_stream. */
yy_status yy_radial_scan_static(const double *r_edges, int n_r, int l_max, double G,
                                const double *moments, double *coeff, void *cuda_stream);

/* Number of CUDA kernels the last yy_potential call launched (-1 for NULL). */
int yy_last_launch_count(const yy_grid *g);

/* Flop count of one solve with the analysis evaluation of the last solve
 * (2 M N K dense, or its two separable stages; dense before the first solve),
 * the moment combination, and one or four synthesis
 * contractions (with_gradient = 0 / 1; K = n_lm each), in floating-point
 * operations (the algorithmic count, before any operand splitting). */
double yy_solve_flops(const yy_grid *g, int with_gradient);

/* ---- batched solves ------------------------------------------------------
 * Many independent density fields, each on its own grid (uneven n_r, angular
 * resolution and l_max), solved by one CUDA graph.  A field is described by
 * the arguments of yy_grid_create; the batch owns one grid per field. */
typedef struct yy_batch yy_batch;
typedef struct {
  const double *r_edges;       /* host, n_r + 1 values (copied) */
  int n_r, n_theta, n_phi;
  double delta_theta, delta_phi;
  int l_max;
  double G;
} yy_field_desc;

/* Create the fields' grids (rules and errors of yy_grid_create, per field;
 * 1 <= n_fields <= 65536).  Synchronises.  *out is NULL on failure. */
yy_status yy_batch_create(const yy_field_desc *fields, int n_fields, yy_batch **out);

/* yy_grid_prepare for every field. */
yy_status yy_batch_prepare(yy_batch *b, yy_precision prec);

/* Autotuner: for every field, time each evaluation (YY_ANALYSIS_DENSE,
 * YY_ANALYSIS_SEPARABLE; reps solves each on zero densities in scratch
 * buffers it allocates and frees) in the given form, with or without the
 * gradient, together with the K split of the dense tensor-core analysis
 * (half the default and the default, which is also the largest; the
 * results do not depend on it, see yy_grid_set_analysis_splits), and
 * record the fastest for that form: later graphs of that form use it (other
 * forms keep theirs; untuned forms use YY_ANALYSIS_AUTO and the rule).  The
 * first yy_batch_potential after tuning also times its graph with 1, 2, 4, 8
 * and 16 parallel branches on the caller's buffers, keeps the fastest, and
 * synchronises.  chosen (NULL or n_fields entries) receives the yy_analysis
 * picked per field.  Prepares the form; synchronises.  The separable
 * tensor-core tables of this form are freed for fields that pick the dense
 * evaluation, and rebuilt (before any capture) if a field is later set to
 * YY_ANALYSIS_SEPARABLE. */
yy_status yy_batch_tune(yy_batch *b, yy_precision prec, int with_gradient, int reps, int *chosen);

/* Set one field's analysis evaluation by hand, for every form (see
 * yy_analysis). */
yy_status yy_batch_set_analysis(yy_batch *b, int field, yy_analysis method);

/* Solve every field.  Each argument is a host array of n_fields device
 * pointers laid out as for yy_potential; grad_yin and grad_yang are both NULL
 * (no gradient) or both arrays.  The first call with a given set of pointers,
 * form and gradient flag records all solves into one CUDA graph (fields on
 * parallel branches) and instantiates it; later calls with the same set replay
 * it on cuda_stream (one graph launch, bitwise-identical results).  A few
 * graphs are kept.  Asynchronous.  Errors as for yy_potential. */
yy_status yy_batch_potential(yy_batch *b, const double *const *rho_yin, const double *const *rho_yang,
                             double *const *phi_yin, double *const *phi_yang,
                             double *const *grad_yin, double *const *grad_yang,
                             yy_precision prec, void *cuda_stream);

/* The grid of one field (owned by the batch; NULL if out of range). */
yy_grid *yy_batch_grid(yy_batch *b, int field);

/* Kernels in the graph the last yy_batch_potential launched (-1 for NULL). */
int yy_batch_last_launch_count(const yy_batch *b);

/* Grouped solves: `groups` concurrent groups of fields, or 0 for one graph
 * of per-field solves (default: grouped, two groups).  In a tensor-core form, when every field
 * uses the dense evaluation (YY_ANALYSIS_AUTO or _DENSE, as yy_batch_tune
 * records for the batched workload) and fits the grouped kernels (two
 * patches, l_max <= 80, n_r <= 768, rows of at most 24,576 cells and 2,048
 * modes), the graph holds one launch per stage over all fields: the density
 * packing, the analysis contraction (one tile list spanning every field's
 * tiles, each field's tensor maps in device memory), the split-K sum with
 * the patches' combination, the radial scans, the coefficient packing and the
 * synthesis contraction -- six to eight kernels (the density rows take the
 * form the field's own solve packs them in: a warp a row up to 2,048 cells,
 * streamed when longer and even, a block a row otherwise), with each field's
 * arithmetic that of its own solve (bitwise the same results).  The fields
 * are split into groups of about equal work that run side by side, each with
 * its own launch per stage; unless this call fixed their number, the first
 * grouped capture after yy_batch_tune times one, two and four groups and
 * keeps the fastest.  Otherwise, or with groups = 0, every field's solve is
 * recorded on parallel branches.  The call drops the recorded graphs.
 * Errors: YY_ERR_INVALID_ARG for NULL or groups outside 0 .. 16. */
yy_status yy_batch_set_grouping(yy_batch *b, int groups);

/* Parallel branches of the batch's graphs: 4, or the count the first capture
 * after yy_batch_tune picked by timing 1, 2, 4, 8 and 16 (-1 for NULL). */
int yy_batch_branches(const yy_batch *b);

/* Concurrent groups of the grouped solves (see yy_batch_set_grouping; 0 when
 * grouping is off, -1 for NULL). */
int yy_batch_groups(const yy_batch *b);

/* K split of the dense tensor-core analysis recorded for a field and form by
 * yy_batch_tune (0: the rule's count; -1 for bad arguments). */
int yy_batch_analysis_splits(const yy_batch *b, int field, yy_precision prec);

/* The first non-OK device status over the fields (reads and clears each). */
yy_status yy_batch_last_device_status(yy_batch *b);

/* Release the batch and its grids (NULL-safe; synchronises). */
void yy_batch_destroy(yy_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* YY_H */
