/*
 * coro.h -- C ABI of libcoro: coronagraph wavefront propagation on one GB300 (sm_103a).
 *
 * The operations follow Douglas & Perrin, "Accelerated Modeling of Near and Far-Field
 * Diffraction for Coronagraphic Optical Systems" (SPIE 2018):
 *   - a sampled complex wavefront built from pupil size, oversampling and wavelength
 *     (Sec. 1.1 "general complex wavefront class"; App. A),
 *   - optical elements multiplied onto it: A exp(2 pi i OPD / lambda) (Eq. 3), thin lenses
 *     and quadratic phase factors exp(i pi r^2 / (lambda z)) (Eq. 2; Sec. 1.1),
 *   - plane-to-plane Fresnel propagation by the angular-spectrum and direct methods
 *     (Sec. 1.1, Sec. 2.2),
 *   - the matrix Fourier transform of the semi-analytic coronagraph method (Sec. 1.1, Sec. 2.3),
 *   - detector intensity and dark-hole reductions (Sec. 1, the 1e-10 contrast goal).
 *
 * Conventions (the paper states none of them):
 *   - A field is [batch][n][n] interleaved complex (re, im), row-major [y][x], in DEVICE
 *     memory owned by the caller. CORO_C64 = float2, CORO_C128 = double2.
 *   - Pixel centres sit at x_j = (j - n/2) * pixelscale; the optical axis is pixel n/2.
 *   - DFT sign: forward exp(-2 pi i jk/n); inverse carries 1/n per axis.
 *   - SI units (metres, radians); focal-plane sampling in lambda/D per pixel.
 *
 * Every call returns a coro_status and never aborts the process. Arguments are checked on the
 * host before any launch; on failure nothing is launched and coro_last_error() (thread-local)
 * describes the problem. All launches are asynchronous on the context's stream; device
 * pointers handed in are borrowed for the duration of that stream-ordered work. There is no
 * CPU fallback: without a CUDA device every call that launches work returns CORO_ECUDA.
 */
#ifndef CORO_H
#define CORO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CORO_VERSION 1

typedef enum {
    CORO_OK = 0,
    CORO_EINVAL = -1,     /* bad argument (null pointer, unsupported size, bad enum)        */
    CORO_ENOMEM = -2,     /* device or host allocation failed                               */
    CORO_ECUDA = -3,      /* a CUDA runtime call failed (message in coro_last_error)        */
    CORO_ETIMEOUT = -4,   /* a bounded device-side wait expired (status flag set by kernel) */
    CORO_ENOTIMPL = -5,   /* combination not implemented                                    */
    CORO_ESIZE = -6       /* size outside the supported range                               */
} coro_status;

typedef enum { CORO_C64 = 0, CORO_C128 = 1 } coro_dtype;

/* ------------------------------------------------------------------------------------------
 * Context: one device, one stream, cached twiddle tables.
 * ------------------------------------------------------------------------------------------ */
typedef struct coro_ctx_s* coro_ctx;

/* Create a context on `device` issuing work on `stream` (a cudaStream_t, borrowed; NULL =
 * legacy default stream). Allocates small device tables lazily. *out owned by the caller,
 * released by coro_ctx_destroy. Errors: CORO_EINVAL (out NULL), CORO_ECUDA (no device). */
coro_status coro_ctx_create(int device, void* stream, coro_ctx* out);
coro_status coro_ctx_destroy(coro_ctx ctx);
/* Change the stream later launches go to (borrowed). */
coro_status coro_ctx_set_stream(coro_ctx ctx, void* stream);
/* Block the host until the context's stream has drained; reports asynchronous faults. */
coro_status coro_ctx_synchronize(coro_ctx ctx);
/* Failure-path self-test (no counterpart in the paper): launches one thread that waits, for at
 * most `polls` (1 .. 2^20) polls, on an mbarrier nothing completes. The bounded wait expires
 * as a stalled copy or MMA would, sets the context's error flag and returns; the next
 * coro_ctx_synchronize reports CORO_ETIMEOUT (and clears the flag), and the context stays
 * usable. No fault, trap or hang is involved. */
coro_status coro_selftest_wait_timeout(coro_ctx ctx, int polls);
/* Thread-local description of the last failure ("" if none). Valid until the next call. */
const char* coro_last_error(void);
int coro_version(void);

/* ------------------------------------------------------------------------------------------
 * Wavefront descriptor (Sec. 1.1 complex wavefront class; App. A FresnelWavefront).
 * Plain struct; no memory is owned by the library.
 *   data        device, [batch][n][n] complex (see dtype), row-major [y][x]
 *   pixelscale  host, [batch], metres per pixel; the direct Fresnel hop rewrites it
 *   wavelength  host, [batch], metres
 * n is a power of two in [32, 8192] (C128: [32, 4096]); batch >= 1.
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    void* data;
    int dtype;
    int batch;
    int n;
    double* pixelscale;
    const double* wavelength;
} coro_wavefront;

/* a1: fill every sample with `amplitude` (App. A: a new wavefront has unit amplitude). */
coro_status coro_wavefront_init(coro_ctx ctx, const coro_wavefront* wf, double amplitude);
/* y <- y + alpha x, sample by sample, for two wavefronts of the same dtype, batch and n (alpha
 * real). Used for Babinet's principle when a coronagraph is composed from single calls
 * (E_C = E_A - IMFT(spot . MFT(E_A)), Sec. 1.1). */
coro_status coro_wavefront_axpy(coro_ctx ctx, double alpha, const coro_wavefront* x, const coro_wavefront* y);

/* ------------------------------------------------------------------------------------------
 * Optical elements (a2, a3). An element multiplies the field pointwise by a transmission.
 * Geometry uses the wavefront's per-item pixelscale (metres) unless noted.
 * ------------------------------------------------------------------------------------------ */
typedef enum {
    CORO_EL_APERTURE = 1, /* circular aperture r <= radius, central obscuration r < obscuration
                             * radius, n_spiders (0 or 4) vanes |x|<w/2 or |y|<w/2 (App. A
                             * CircularAperture; obscured/spidered pupils)                    */
    CORO_EL_CIRCLE = 2,   /* circular stop r <= radius transmits; CORO_ELF_OPAQUE_INSIDE makes
                             * it an occulting spot (field stops, Lyot stops, occulters)      */
    CORO_EL_LENS = 3,     /* thin lens exp(-i pi r^2 / (lambda f)) (Sec. 1.1, Eq. 2 reading)  */
    CORO_EL_OPD_MAP = 4,  /* A exp(2 pi i OPD / lambda) from a device float map (Eq. 3);
                             * amplitude map optional                                         */
    CORO_EL_ZERNIKE = 5,  /* OPD = sum_j c_j Z_j(r/radius) over Noll j = j_first.., zero
                             * outside the disk (unit-RMS Noll normalisation)                 */
    CORO_EL_SINE = 6,     /* OPD = sine_amplitude * sin(2 pi sine_freq x) along x (axis 0) or y
                             * (axis 1) (App. A SineWaveWFE)                                   */
    CORO_EL_SCALAR = 7,   /* multiply by a real scalar (ScalarTransmission, App. B)            */
    CORO_EL_CHECKPOINT = 8, /* copy the field as it stands at this point of the plane (after the
                             * plane's elements listed before it) to `store`, field unchanged:
                             * per-plane wavefront checkpoints for adjoints (intermediate planes
                             * of Sec. 1.1 systems). store: device, the wavefront's dtype,
                             * [batch][n][n]; it must stay allocated for the plan's life and is
                             * also written while a plan is tuned at creation. In pilot-beam
                             * systems the copy is the field relative to the plane's reference
                             * surface, as the plane's other elements see it.                 */
    CORO_EL_PHASE_GRAD = 9 /* adjoint tap: with the field holding the adjoint G = dL/dconj(E)
                             * and `ref` the forward field E at the same point, writes the
                             * float map store[b][y][x] = (scalar / lambda_b) * 2 Im(G conj(E)),
                             * i.e. scalar / lambda_b times dL/dphi of a phase exp(i phi) applied
                             * there (scalar = 4 pi: dL/dh per metre of a reflecting surface
                             * at normal incidence). Field unchanged. ref: device, the
                             * wavefront's dtype, [batch][n][n], or NULL for a unit reference
                             * (E = 1: the tap after the conjugate of a known transmission
                             * recomputes that plane instead of reading a checkpoint);
                             * store: device float [batch][n][n]. Same placement rules as
                             * CHECKPOINT.                                                    */
} coro_element_kind;

#define CORO_ELF_OPAQUE_INSIDE 1  /* CORO_EL_CIRCLE: block r <= radius instead of passing it */
#define CORO_ELF_MAP_BATCHED   2  /* CORO_EL_OPD_MAP: map is [batch][n][n], else [n][n]       */

typedef struct {
    int kind;                 /* coro_element_kind                                           */
    int flags;                /* CORO_ELF_*                                                  */
    int plane;                /* plane index inside a Fresnel plan (ignored by apply_element) */
    int n_spiders;            /* APERTURE: 0 or 4                                            */
    double radius;            /* APERTURE/CIRCLE/ZERNIKE: metres                             */
    double obscuration;       /* APERTURE: fraction of radius (0 = none)                     */
    double spider_width;      /* APERTURE: vane width, metres                                */
    double focal_length;      /* LENS: metres (positive = converging)                        */
    const float* opd;         /* OPD_MAP: device, metres                                     */
    const float* amplitude;   /* OPD_MAP: device amplitude (same shape as opd) or NULL       */
    const double* coeffs;     /* ZERNIKE: host, metres, n_coeffs values                      */
    int j_first;              /* ZERNIKE: Noll index of coeffs[0] (>= 1)                     */
    int n_coeffs;             /* ZERNIKE: count, j_first + n_coeffs - 1 <= 36                */
    double sine_freq;         /* SINE: cycles per metre                                      */
    double sine_amplitude;    /* SINE: metres                                                */
    int axis;                 /* SINE: 0 = varies along x, 1 = along y                       */
    double scalar;            /* SCALAR                                                      */
    void* store;              /* CHECKPOINT / PHASE_GRAD: device destination [batch][n][n]   */
    const void* ref;          /* PHASE_GRAD: device forward field [batch][n][n]              */
} coro_element;

/* Apply one element in place (unfused elementwise kernel). */
coro_status coro_apply_element(coro_ctx ctx, const coro_wavefront* wf, const coro_element* el);

/* ------------------------------------------------------------------------------------------
 * Fresnel propagation (a4-a6, a6').
 * CORO_FRESNEL_AS: angular spectrum (Sec. 1.1, Lawrence Eqs. 82-89 cited):
 *     E(z) = IDFT2[ exp(-i pi lambda z (fx^2 + fy^2)) DFT2[E] ], pixelscale unchanged.
 * CORO_FRESNEL_DIRECT: single-FFT Fresnel (Sec. 1.1):
 *     E'(u) = 1/(i lambda z) exp(i pi u^2/(lambda z)) dx^2 sum_x E(x) exp(i pi x^2/(lambda z))
 *             exp(-2 pi i x u/(lambda z)) on the grid u_k = (k - n/2) du,
 *     pixelscale[b] <- du = |lambda_b z / (n dx_b)| (a forward DFT for z > 0, the unscaled
 *     inverse DFT for z < 0; one more pass for z < 0).
 * DFTs are centred (fftshift folded into the kernels). The global piston exp(2 pi i z/lambda)
 * is dropped. z != 0. Three HBM passes (row FFT, column FFT*H*IFFT, row IFFT).
 * ------------------------------------------------------------------------------------------ */
typedef enum { CORO_FRESNEL_AS = 0, CORO_FRESNEL_DIRECT = 1 } coro_fresnel_method;

coro_status coro_propagate_fresnel(coro_ctx ctx, coro_wavefront* wf, double z, int method);

/* Centred 2-D DFT in place: direction -1 forward (no scaling), +1 inverse (1/n^2). Used for
 * Fraunhofer propagation by large FFT (Sec. 1.1). */
coro_status coro_fft2(coro_ctx ctx, const coro_wavefront* wf, int direction);

/* ------------------------------------------------------------------------------------------
 * Fused Fresnel system (D2: the ordered (optic, distance) list of App. B).
 * Plane p receives every element whose .plane == p (applied in array order), then the field
 * hops distance[p] by method[p] to plane p+1 (for p < n_planes-1). Consecutive hops are fused
 * so that each angular-spectrum hop costs two HBM round trips: a row pass
 * (IFFT_rows . elements . FFT_rows) and a column pass (FFT_cols . H . IFFT_cols).
 * flags: CORO_PLAN_INIT_UNIFORM -- the input is a unit-amplitude field (a1) that is generated
 * in the first pass instead of read.
 * The plan copies everything it needs (tables are built on the device in FP64 and rounded to
 * the field precision), except device maps referenced by elements, which must stay valid and
 * unchanged while the plan is executed.
 * ------------------------------------------------------------------------------------------ */
#define CORO_PLAN_INIT_UNIFORM 1

typedef struct coro_plan_s* coro_plan;

typedef struct {
    int dtype;
    int batch;
    int n;
    const double* pixelscale;   /* host [batch], pixelscale at plane 0                       */
    const double* wavelength;   /* host [batch]                                              */
    int n_planes;
    const double* distance;     /* host [n_planes-1], metres                                 */
    const int* method;          /* host [n_planes-1], coro_fresnel_method; NULL = all AS     */
    int n_elements;
    const coro_element* elements;
    int flags;
} coro_fresnel_desc;

coro_status coro_fresnel_plan_create(coro_ctx ctx, const coro_fresnel_desc* desc, coro_plan* out);
/* f2: a Fresnel system with the propagation method chosen automatically (Sec. 1.1: the
 * angular-spectrum / direct choice the paper takes from Lawrence; POPPY's Fresnel wavefront).
 * A Gaussian pilot beam with waist `beam_radius` at plane 0 is carried through the system by
 * its complex parameter q (q += d per hop; 1/q -= 1/f per CORO_EL_LENS). A plane is inside
 * when |Re q| < |Im q| (within one Rayleigh distance of the pilot waist) and stores the field
 * on a planar reference; outside planes store it divided by exp(i pi r^2/(lambda R)), R = Re q
 * (the distance from the pilot waist). Hops: inside -> inside angular spectrum; inside ->
 * outside angular spectrum to the waist, then a direct hop without output quadratic phase;
 * outside -> inside a direct hop without input quadratic phase to the waist, then angular
 * spectrum; outside -> outside two direct hops through the waist. Direct hops change the pixel
 * scale (|lambda z/(n dx)|); a direct hop with z < 0 is the inverse DFT, keeping the natural
 * orientation. Lenses become quadratic phases that also swap the reference surface. The last
 * plane's field is returned on a planar reference. Decisions are made per item and must agree
 * across the batch (else CORO_ENOTIMPL). The result is a Fresnel plan (execute, pass info,
 * graphs, timing apply); pixelscale_out of execute gives the final pitch. */
typedef struct {
    int dtype;
    int batch;
    int n;
    const double* pixelscale;   /* host [batch], pixelscale at plane 0                       */
    const double* wavelength;   /* host [batch]                                              */
    double beam_radius;         /* pilot-beam waist radius at plane 0, metres (> 0)          */
    int n_planes;
    const double* distance;     /* host [n_planes-1], metres, finite and nonzero             */
    int n_elements;
    const coro_element* elements;   /* CORO_EL_LENS elements also refocus the pilot beam     */
    int flags;                  /* CORO_PLAN_INIT_UNIFORM                                    */
} coro_fresnel_system_desc;

coro_status coro_fresnel_system_create(coro_ctx ctx, const coro_fresnel_system_desc* desc, coro_plan* out);
/* For a plan made by coro_fresnel_system_create: spherical (host [n_planes], may be NULL)
 * receives 1 for planes outside the pilot beam's Rayleigh range, *direct_hops the number of
 * direct sub-hops. */
coro_status coro_fresnel_system_info(coro_plan plan, int* spherical, int* direct_hops);
/* pitch (host [batch]): the pixel scale (metres) at which plane `plane`'s elements act, per
 * item -- for masks generated on the host at planes whose sampling the plan chose (a focal
 * plane mask behind a direct hop). Works for any Fresnel plan. */
coro_status coro_fresnel_system_pitch(coro_plan plan, int plane, double* pitch);

/* Run the plan in place on `field` (device, [batch][n][n]). pixelscale_out (host [batch], may
 * be NULL) receives the final pixel scale. */
coro_status coro_fresnel_plan_execute(coro_plan plan, void* field, double* pixelscale_out);
/* `times` executes back to back on the same field (one graph when graphs are on): the
 * repeated-system throughput measurement, with per-pass timing when enabled. */
coro_status coro_fresnel_plan_execute_n(coro_plan plan, void* field, int times);
/* Number of kernels one execute launches (for launch accounting). */
coro_status coro_plan_launch_count(coro_plan plan, int* out);
/* Run passes [first, first + count) of the plan only (for per-launch timing); ranges always
 * run every pass in place on the natural layout, so running every range in order matches
 * coro_fresnel_plan_execute exactly for a plan on the natural layout and up to FP32 rounding
 * order for one on the alternating layout (coro_fresnel_plan_set_layout). */
coro_status coro_fresnel_plan_execute_range(coro_plan plan, void* field, int first, int count);
/* Describe pass i: *is_row (1 = row pass, 0 = column pass) and *bytes, the algorithmic HBM
 * traffic of the launch (field read unless generated, field write, OPD/amplitude maps read). */
coro_status coro_fresnel_plan_pass_info(coro_plan plan, int i, int* is_row, double* bytes);
/* *flops: the pass's line transforms at the conventional 5 N log2 N real flops each (N lines
 * per item, one or two transforms per pass), elements and tables not counted. */
coro_status coro_fresnel_plan_pass_flops(coro_plan plan, int i, double* flops);
/* Kernel that pass i launches, as chosen when the plan was built (the complex64 plan times
 * its candidates then unless the environment sets CORO_AUTOTUNE=0). *persistent:
 *   0  one block per group of lines;
 *   1  persistent kernel: one block per SM slot, line groups staged through shared memory
 *      by bulk or TMA copies while the previous group is transformed;
 *   2  unit-pipelined persistent kernel: one block per SM split into independent units
 *      with their own barriers, sharing staged line groups;
 *   3  as 2, each unit transforming two lines (columns, or rows) at once in packed FP32x2
 *      arithmetic;
 *   4  wide kernel: four-column groups (32-byte row segments) staged by TMA, packed FP32x2
 *      arithmetic, half-size exchange buffers, results stored from registers.
 * *lines = columns per group for a column pass, 0 for a row pass. Either output pointer may
 * be NULL. Plain host query; no device work. */
coro_status coro_fresnel_plan_pass_kernel(coro_plan plan, int i, int* persistent, int* lines);
/* (*persistent 6: mixed-radix kernels for n not a power of two; 7: the packed-pair kernels of
 * the alternating layout, below; 8: quad kernel, four-column strips (whole 32-byte sectors)
 * as two packed pairs, streamed by TMA in quarter strips, exchanges in swizzled shared
 * memory of exactly N slots per pair; 9: mixed-radix packed-pair kernels, two lines per block
 * in packed FP32x2 arithmetic with the radix plan fixed at compile time, in place in one
 * shared buffer, for the lengths built in (1400, 2800, 4100).) */
/* Radix sequence of pass i's line transforms (the FFT factorisation the chosen kernel runs):
 * radices[0 .. min(*stages, max_radices) - 1], *stages the number of stages (radices may be
 * NULL when max_radices is 0). Register-resident engines: radix 16 while it divides, the
 * remainder last (4096 = 16 x 16 x 16); the shared-memory engine: mixed_plan's sequence
 * (2800 = 16 x 5 x 5 x 7; row variant 5 / column lines -8 at a power of two: radix 8,
 * 4096 = 8 x 8 x 8 x 8). Plain host query. */
coro_status coro_fresnel_plan_pass_radix(coro_plan plan, int i, int* radices, int max_radices, int* stages);
/* Override the tuned kernel choice of every pass of a complex64 plan.
 *   row_variant: 0 persistent, 1 one block per line group, 2 unit-pipelined, 3 packed row
 *                pairs, 5 the shared-memory engine with radix 8 (2, 3 and 5: N = 1024 ...
 *                4096); at mixed-radix N: 0 the shared-memory engine, 6 the packed-pair
 *                engine (N = 1400, 2800, 4100).
 *   col_lines:   columns per block (a width the plan's N supports), -1 persistent TMA,
 *                -2 unit-pipelined, -3 packed column pairs, -4 wide, -7 quad, -8 the
 *                shared-memory engine with radix 8 (-2 to -8: N = 1024 ... 4096), 0 default;
 *                at mixed-radix N: columns per block of the shared-memory engine, or -5 the
 *                packed-pair engine (N = 1400, 2800, 4100).
 * Values the plan's N does not offer are rejected with CORO_EINVAL and nothing changes.
 * Every choice gives the same result up to FP32 rounding order (used to test each kernel). */
coro_status coro_fresnel_plan_set_pass_kernel(coro_plan plan, int row_variant, int col_lines);
/* (set_pass_kernel also returns the plan to the natural layout.)
 * Plane layout between passes (complex64 plans, n = 1024, 2048, 4096). Natural (0): every
 * pass transforms the field in place, column passes reading and writing strided column
 * pairs. Alternating (1): a column pass followed by a row pass writes its result transposed
 * ([b][x][y], contiguous rows) into a plane the plan owns (batch x n x n complex64, allocated
 * here, freed on return to 0 or with the plan), and the row pass reads it back column-wise
 * and writes the field's rows; each pass then has one strided side. Results agree up to FP32
 * rounding order. At creation the plan times both and keeps the faster (natural when
 * CORO_AUTOTUNE=0) unless the environment sets CORO_LAYOUT=0 (natural) or CORO_LAYOUT=1
 * (alternating). CORO_ENOTIMPL: the plan has no column pass followed by a row pass at a
 * supported size. */
coro_status coro_fresnel_plan_set_layout(coro_plan plan, int transposed);
/* Give dst the kernel choices and layout the tuner made for src (plans of the same dtype, n,
 * batch and pass sequence, e.g. a second buffer slot of one system): the two then run the
 * same kernels. CORO_EINVAL when they differ; dst is unchanged then. */
coro_status coro_fresnel_plan_copy_tuning(coro_plan dst, coro_plan src);
coro_status coro_fresnel_plan_layout(coro_plan plan, int* transposed);
/* a10: replay plan execution as one CUDA graph (enable = 1) or launch kernel by kernel (0,
 * the default). With graphs on, the first execute with a given set of device pointers
 * (field; or pupil, intensity and field) runs eagerly and captures its launch sequence on a
 * private stream; later executes with the same pointers replay it on the context's stream,
 * and new pointers trigger a new capture. Host-side arguments (the Lyot peak normalisation)
 * are copied to the device before each replay, outside the graph. Results are identical to
 * the eager path. execute_range and the gradient never use the graph. */
coro_status coro_plan_set_graph(coro_plan plan, int enable);
/* Per-unit timing (units: the passes of a Fresnel plan; the six stages of execute_range for a
 * Lyot plan). steps > 0 creates steps x (units + 1) CUDA events: the k-th execute of an
 * execute_n call (execute counts as k = 0) records set k before its first unit and after
 * every unit, on the stream the kernels run on and inside the graph when one is replayed.
 * steps = 0 releases them. Synchronises the device; drops a captured graph. */
coro_status coro_plan_set_timing(coro_plan plan, int steps);
/* ms (host, [steps][units]): unit durations of executes 0..steps-1 of the last timed call
 * (steps <= the count given to coro_plan_set_timing; every one of them must have run).
 * Waits for the last of those events. */
coro_status coro_plan_unit_times(coro_plan plan, int steps, float* ms);
coro_status coro_plan_destroy(coro_plan plan);

/* ------------------------------------------------------------------------------------------
 * Matrix Fourier transform (a7; Sec. 1.1 "discrete matrix Fourier transforms", Soummer 2007;
 * Sec. 2.3 "sines and cosines ... in the matrix DFT").
 * direction -1 (pupil -> focal plane):
 *     out[v,u] = s sum_{i,j} in[i,j] exp(-2 pi i (X_j U_u + Y_i V_v)),
 *     X_j = (j - n/2)/npix (units of D), U_u = (u - m/2) du (units of lambda/D), s = du/npix.
 * direction +1 (focal plane -> pupil): input pitch du (lambda/D), output pitch 1/npix (D),
 *     exponent +2 pi i, same s.
 * in: [batch][n_in][n_in]; out: [batch][m][m], both C64 (precisions FP32 / 3XTF32 / 3XBF16 / EXT) or
 * both C128 (precision FP64). du: host [batch] (lambda/D per pixel of the focal-plane side).
 * npix: pupil pixels across D. precision: coro_mft_prec.
 * Work buffers are taken from the context (allocated on first use, grown as needed).
 * ------------------------------------------------------------------------------------------ */
typedef enum {
    CORO_MFT_FP32 = 0,    /* FP32 CUDA-core complex GEMM                                     */
    CORO_MFT_3XTF32 = 1,  /* split TF32 tensor-core GEMM (hi*hi + hi*lo + lo*hi), FP32 acc   */
    CORO_MFT_3XBF16 = 2,  /* split BF16 tensor-core GEMM, FP32 accumulate                    */
    CORO_MFT_FP64 = 3,    /* complex128 fields, FP64 CUDA-core GEMM (reference precision)    */
    CORO_MFT_EXT = 4      /* extended precision on the BF16 tensor cores: each operand value  */
                          /* as four 8-bit slices of a power-of-two scale shared by 32       */
                          /* consecutive K elements (32 bits), ten slice products summed     */
                          /* exactly per 32-element group, two-float accumulation across     */
                          /* groups and in the epilogues; complex64 in and out               */
} coro_mft_prec;

coro_status coro_propagate_mft(coro_ctx ctx, const coro_wavefront* in, double npix, int direction,
                               int m, const double* du, int precision, coro_wavefront* out);

/* ------------------------------------------------------------------------------------------
 * Deformable mirror (Sec. 1.2: 32x32 / 48x48-actuator DMs sampled by hundreds of pixels).
 * Gaussian influence g(d) = exp(-d^2/(2 sigma^2)), sigma = fwhm / (2 sqrt(2 ln 2)); actuator
 * centres (q - (na-1)/2) * pitch, pixel centres (x - n/2) * pixelscale (metres).
 * coro_dm_opd:       opd[b][y][x]  = scale * sum_{p,q} heights[b][p][q] g(y - y_p) g(x - x_q)
 *                    (scale = 2 for the reflected OPD of a surface), device float arrays.
 * coro_dm_correlate: grad[b][p][q] = scale * sum_{y,x} w[b][y][x] g(y - y_p) g(x - x_q), the
 *                    transpose of coro_dm_opd (gradient of a loss w.r.t. heights from its
 *                    gradient w.r.t. the OPD map). Terms below 1e-20 of the peak are skipped.
 * ------------------------------------------------------------------------------------------ */
coro_status coro_dm_opd(coro_ctx ctx, const float* heights, int batch, int na, double pitch, double fwhm,
                        int n, double pixelscale, double scale, float* opd);
coro_status coro_dm_correlate(coro_ctx ctx, const float* w, int batch, int n, double pixelscale, int na,
                              double pitch, double fwhm, double scale, float* grad);

/* ------------------------------------------------------------------------------------------
 * Batched semi-analytic Lyot coronagraph (a7-a10; Sec. 1.1: the Soummer et al. method of
 * matrix Fourier transforms around a small focal-plane mask), per item b:
 *   E_B   = MFT(E_A; m_occ, du_occ)                      pupil -> occulter
 *   E_C   = E_A - MFT^-1(spot . E_B)                      Babinet; spot = 1 for rho <= spot_radius
 *   E_D   = E_C . Lyot stop (r <= lyot_frac * D/2)
 *   E_det = MFT(E_D; m_det, du_det)
 *   I = |E_det|^2 / peak[b],   S[b] = sum of I over dh_in <= rho <= dh_out (lambda/D)
 * MFT conventions as in coro_propagate_mft (pupil pixel centre n/2, npix pixels across D).
 * Six split-precision tensor-core GEMMs over the whole batch; spot, Babinet subtraction, Lyot
 * stop, intensity and dark-hole sum are fused into GEMM epilogues. Items may have different
 * occulter sizes m_occ (uneven per-wavelength sampling); n, npix, lyot_frac, m_det are shared.
 * The plan owns its work buffers (bases, split operands, about 80 MB per item at n = 1024 with
 * TF32) for its lifetime.
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    int m_occ;            /* occulter samples per axis, [16, 8192]                          */
    double du_occ;        /* lambda/D per occulter pixel                                     */
    double spot_radius;   /* occulting spot radius, lambda/D                                 */
    double du_det;        /* lambda/D per detector pixel                                     */
    double dh_in, dh_out; /* dark-hole annulus, lambda/D (inclusive)                         */
} coro_lyot_item;

typedef struct {
    int batch;
    int n;                /* pupil array n x n, [16, 8192]                                   */
    double npix;          /* pupil pixels across D                                           */
    double lyot_frac;     /* Lyot stop radius / pupil radius                                 */
    int m_det;            /* detector samples per axis                                       */
    const coro_lyot_item* items;  /* host [batch], copied                                    */
    int precision;        /* CORO_MFT_3XTF32, CORO_MFT_3XBF16 or CORO_MFT_EXT (complex64     */
                          /* pupils; EXT keeps the peak and 1/peak in FP64); or CORO_MFT_FP64: the same  */
                          /* chain item by item on complex128 pupils/fields with FP64 MFTs  */
                          /* (exact to FP64 rounding; execute, execute_n and peak only --    */
                          /* execute_range, gradient and set_pupil_layout return            */
                          /* CORO_ENOTIMPL; flops reports 0 tensor flops; executes are not   */
                          /* replayed as graphs)                                             */
} coro_lyot_desc;

coro_status coro_lyot_plan_create(coro_ctx ctx, const coro_lyot_desc* desc, coro_plan* out);
/* pupil: device complex64 [batch][n][n] (E_A; complex128 for CORO_MFT_FP64). peak: host [batch]
 * normalisation (NULL = 1). intensity: device float [batch][m_det][m_det] or NULL. field: device
 * complex64 (complex128 for CORO_MFT_FP64) [batch][m_det][m_det] (unnormalised E_det) or NULL. dh: host [batch] dark-hole sums or NULL
 * (when given, the stream is synchronised). */
coro_status coro_lyot_plan_execute(coro_plan plan, const void* pupil, const double* peak, float* intensity,
                                   void* field, double* dh);
/* `times` executes back to back (one graph when graphs are on), without the host copy of dh;
 * per-stage timing when enabled. */
coro_status coro_lyot_plan_execute_n(coro_plan plan, const void* pupil, const double* peak, float* intensity,
                                     void* field, int times);
/* Normalisation: peak_out[b] = max |E_det|^2 of the same chain with the occulter removed
 * (E_D = E_A . Lyot stop). Synchronises the stream. */
coro_status coro_lyot_plan_peak(coro_plan plan, const void* pupil, double* peak_out);
/* Run stages [first, first + count) only (for per-launch timing): 0 split of the pupil, 1-4 the
 * GEMMs pupil->occulter (two), occulter->Lyot with Babinet (two), 5 the detector MFT with the
 * intensity epilogue (two launches, preceded by one stream memset of the dark-hole sums).
 * Running 0-5 in order equals coro_lyot_plan_execute without the host copy of dh. */
coro_status coro_lyot_plan_execute_range(coro_plan plan, const void* pupil, const double* peak, float* intensity,
                                         void* field, int first, int count);
/* Tensor work of one execute (the six GEMMs), in flops: *useful = 24 per valid output per
 * complex product inside the operands' known support (the spot, the Lyot stop: the plan runs
 * only the K ranges and tiles those leave non-zero); *issued = the same over every 128 x 128
 * tile and K slice the kernels run (padding included). Either pointer may be NULL. Host only. */
coro_status coro_lyot_plan_flops(coro_plan plan, double* useful, double* issued);
/* Tensor-core GEMM output tile of the plan (rows x complex columns): 128 x 128 for 3XTF32 /
 * 3XBF16; 128 x 64 or 128 x 32 for EXT, chosen when the plan is created by timing the plan's
 * GEMM stages at both widths (unless the environment sets CORO_AUTOTUNE=0, which keeps 64);
 * 0 x 0 for FP64 plans (CUDA-core GEMMs). Either pointer may be NULL. Host query. */
coro_status coro_lyot_plan_gemm_tile(coro_plan plan, int* tile_m, int* tile_n);
/* Override the tile width: 64 or 32 for EXT plans, 128 (the only one) for 3XTF32 / 3XBF16;
 * other values return CORO_EINVAL and change nothing. Results agree across widths to FP32
 * rounding order. Drops a captured graph. */
coro_status coro_lyot_plan_set_gemm_tile(coro_plan plan, int tile_n);

/* Pupil argument layout for execute / peak / gradient: item b, row i, column j of E_A at
 * pupil[b * bstride + i * ld + j] (default ld = n, bstride = n * n), so the pupil can be the
 * centre window of a larger Fresnel grid. */
coro_status coro_lyot_plan_set_pupil_layout(coro_plan plan, int ld, long long bstride);
/* Adjoint (a11): with S[b] the dark-hole sum and I normalised by peak[b] (held fixed),
 * grad[b] = dS[b]/dconj(E_A[b]) (Wirtinger convention: dS = 2 Re sum conj(grad) dE), i.e. the
 * conjugate-transpose chain  grad = G_C - MFT_occ^H(spot . IMFT_occ^H(G_C)),  G_C = Lyot . MFT_det^H
 * (mask . E_det / peak), with MFT^H = the inverse MFT of the same pitch. Also returns the forward
 * sums in dh_out (host [batch], may be NULL; given -> the stream is synchronised). grad is
 * device complex64 written at grad[b * grad_bstride + i * grad_ld + j] for the n x n window only. */
coro_status coro_lyot_plan_gradient(coro_plan plan, const void* pupil, const double* peak, double* dh_out,
                                    void* grad, int grad_ld, long long grad_bstride);

/* ------------------------------------------------------------------------------------------
 * Differentiable wavefront control (a11). Two Gaussian-influence DMs: DM1 in the pupil plane
 * of an n_fresnel^2 grid (pupil npix pixels across diam_m, centred), DM2 after an angular-
 * spectrum hop z_m (Sec. 1.1); the field hops back -z_m, the centre npix^2 window is the pupil
 * of a batched Lyot chain (one item per wavelength). Loss L = sum_b S[b] with S the dark-hole
 * sum normalised by the peak of the zero-height system (computed once, held fixed).
 * coro_wfc_plan_evaluate: heights device float [2][n_act][n_act] (metres of surface, DM1 then
 * DM2); loss (host) and per_item (host [batch]) optional; grad device float [2][n_act][n_act]
 * = dL/dheights, or NULL for the forward only. Synchronises the stream. The plan holds three
 * resident x n_fresnel^2 complex64 fields (checkpoint E1, work, adjoint).
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    int batch;                    /* wavelengths                                           */
    const double* wavelength;     /* host [batch], metres                                  */
    int n_fresnel;                /* Fresnel grid, power of two                            */
    double diam_m;                /* pupil diameter                                        */
    int npix;                     /* pupil pixels across diam (= Lyot pupil array size)    */
    double z_m;                   /* DM1 -> DM2 distance                                   */
    int n_act;                    /* actuators per axis                                    */
    double act_pitch_m, act_fwhm_m;
    double lyot_frac;
    int m_det;
    const coro_lyot_item* items;  /* host [batch], one Lyot item per wavelength            */
    int precision;                /* CORO_MFT_3XTF32, CORO_MFT_3XBF16 or CORO_MFT_EXT      */
    int max_resident;             /* wavelengths held in HBM at once (3 x 8 n_fresnel^2    */
                                  /* bytes each, 5 x where the Fresnel plans may take the  */
                                  /* alternating layout: n_fresnel 1024 ... 4096); 0 = as  */
                                  /* many as fit in 70 % of the free                       */
                                  /* device memory. The band runs in chunks of that many,  */
                                  /* with the same results (per-item sums in item order).  */
} coro_wfc_desc;

coro_status coro_wfc_plan_create(coro_ctx ctx, const coro_wfc_desc* desc, coro_plan* out);
/* Wavelengths resident at once and the number of chunks the band runs in (either may be NULL). */
coro_status coro_wfc_plan_resident(coro_plan plan, int* resident, int* chunks);
/* Normalisation peaks of the zero-height system (host [batch]); computed on first use. */
coro_status coro_wfc_plan_peak(coro_plan plan, double* peak_out);
coro_status coro_wfc_plan_evaluate(coro_plan plan, const float* heights, double* loss, double* per_item,
                                   float* grad);

/* ------------------------------------------------------------------------------------------
 * Detector reductions (a9).
 * coro_intensity: out[b][y][x] = |E|^2 / norm[b] (norm NULL = 1); out device float.
 * coro_darkhole_sum: host_out[b] = sum over rho in [r_in, r_out] of |E|^2 / norm[b], with
 *     rho = |(x - n/2, y - n/2)| * du[b] in lambda/D; FP64 accumulation. Synchronises the
 *     stream to return the host values.
 * ------------------------------------------------------------------------------------------ */
coro_status coro_intensity(coro_ctx ctx, const coro_wavefront* wf, const double* norm, float* out);
coro_status coro_darkhole_sum(coro_ctx ctx, const coro_wavefront* wf, const double* du,
                              double r_in, double r_out, const double* norm, double* host_out);

/* ------------------------------------------------------------------------------------------
 * Allocation-free dark-hole sum. The paper has no counterpart: this exists for callers that
 * cannot allocate device memory while they run -- a real-time wavefront-control loop that must
 * not see allocator latency or jitter between frames, an application whose device heap is
 * owned by another framework, or a process with a memory budget fixed at start-up.
 * Same result as coro_darkhole_sum (same arguments, no context): the field and host_out
 * belong to the caller; the reduction's scratch (bounds, normalisation, accumulators for up
 * to CORO_NOALLOC_MAX_BATCH items, 32 KiB) is one fixed device array inside the library,
 * held by every GPU that loads it until the process exits. No cudaMalloc/cudaFree or other
 * allocating routine is called.
 *   - Runs on the calling thread's current device and on `stream` (a cudaStream_t of that
 *     device, NULL = legacy default stream); synchronises that stream to return the host
 *     values. A field in another device's memory is rejected with CORO_EINVAL.
 *   - The first call on a device looks up the array's device address (once per device, with
 *     that device current) and keeps it for the life of the process; make that first call
 *     before any stream capture. Resetting the device (cudaDeviceReset, or tearing down its
 *     primary context) after that first call is not supported.
 *   - Every call shares the one array: calls that overlap on the GPU (other threads, other
 *     streams) race and must be serialised by the caller. Each call clears the accumulators
 *     it uses before the reduction.
 *   - batch > CORO_NOALLOC_MAX_BATCH returns CORO_ESIZE with a message; nothing is launched.
 * ------------------------------------------------------------------------------------------ */
#define CORO_NOALLOC_MAX_BATCH 1024
coro_status coro_darkhole_sum_noalloc(const coro_wavefront* wf, const double* du, double r_in,
                                      double r_out, const double* norm, void* stream,
                                      double* host_out);

#ifdef __cplusplus
}
#endif
#endif /* CORO_H */
