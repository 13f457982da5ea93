/* xl — GB300-native differentiable free-space optics (C ABI).
 *
 * The hot path of the differentiable optics simulator of XLuminA (arXiv 2310.08408): free-space
 * propagation of sampled complex fields by scalar / vectorial Rayleigh-Sommerfeld (RS / VRS)
 * and by the chirped z-transform (CZT / VCZT), the optical elements the optimiser tunes (SLM
 * and super-SLM phase masks, thin lenses, polarisers, wave plates), the camera intensity and
 * spot-size losses, the hand-written adjoints of all of them, and Adam.
 * Paper passages: Methods, "Features and performance" (propagators, elements, camera);
 * Methods, "Loss function"; Results and Methods on Adam.
 *
 * Conventions
 *   - Time dependence exp(-i w t): outgoing waves exp(+i k r), k = 2 pi / wavelength.
 *   - Lengths in one unit throughout (micrometres in the tests); wavelength in the same unit.
 *   - A grid samples x_m = x0 + m dx (m < nx), y_n = y0 + n dy (n < ny).
 *   - Complex arrays are interleaved (re, im): complex64 (XL_C64) or complex128 (XL_C128),
 *     row-major [batch][component][ny][nx], x fastest, contiguous.
 *   - Gradients follow g = dL/dRe u + i dL/dIm u, so dL = Re sum conj(g) du.
 *
 * Ownership and streams
 *   - Every field, mask, loss and gradient pointer is caller-owned DEVICE memory unless stated.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default stream).
 *   - The library owns a cache of transfer spectra and chirps keyed by (grid, wavelength, z,
 *     window, precision) and a per-stream workspace; both grow on demand with cudaMalloc and are
 *     released by xl_cache_clear(). Calls that would allocate must not run inside stream
 *     capture: warm them up (same sizes) before capturing a CUDA graph.
 *
 * Environment (read by the library; none is needed)
 *   - XL_CACHE_BYTES: byte cap of the spectrum / chirp cache (default 8 GiB; least recently used
 *     entries are freed above it).
 *   - XL_RS_CHUNK_MB: budget of the RS intermediate planes one chunk of a batch may use (default
 *     2048): the row passes run over a chunk per launch, pass 2 over up to 32 elements per launch.
 *   - XL_P3_TMA=0: RS pass 3 gathers its rows with per-thread asynchronous copies instead of
 *     tiled bulk tensor copies (complex64). Results are bit-identical either way.
 *   - XL_RS_RM=0: the complex64 scalar forward and saved-spectrum adjoint keep the transposing
 *     pass 1 instead of the row-major intermediate gathered by pass 2. Bit-identical either way.
 *   - XL_CZT_RM=0: the complex64 scalar CZT forward (window lengths 256..8192, even window
 *     width) keeps the transposing x pass instead of the row-major intermediate whose columns
 *     the y pass gathers with tiled bulk tensor copies. Bit-identical either way.
 *
 * Errors
 *   - Argument checks happen on the host before any launch and return XL_ERR_ARG or
 *     XL_ERR_UNSUPPORTED with nothing enqueued.
 *   - CUDA failures return XL_ERR_CUDA; allocation failures XL_ERR_NOMEM.
 *   - xl_last_error() returns a thread-local message describing the last failure.
 */
#ifndef XL_H_
#define XL_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t xl_status;
#define XL_OK 0
#define XL_ERR_ARG 1
#define XL_ERR_CUDA 2
#define XL_ERR_NOMEM 3
#define XL_ERR_UNSUPPORTED 4
#define XL_ERR_TIMEOUT 5
#define XL_ERR_NONFINITE 6

/* precision of fields (and of phase masks: float for XL_C64, double for XL_C128) */
#define XL_C64 0
#define XL_C128 1

/* flags */
#define XL_Z_DEVICE 1 /* z (and element parameters) are read from device memory at run time */
/* Backward passes only: the loss is invariant under a constant phase factor on the propagated
 * field (true for camera-intensity losses behind linear optics). dL/dz then leaves out the term
 * Re(ik <g_out, u_out>) of the e^{ikz} rotation, which is zero in exact arithmetic but, computed
 * in single precision, adds rounding noise up to k |g_out| |u_out| to a derivative that is often
 * four orders of magnitude smaller. The distance derivative uses the spectrum of dh/dz - ik h. */
#define XL_PHASE_INVARIANT 2
/* CZT backward calls only: add the field gradient and g_z to what g_in and g_z hold instead of
 * overwriting them (the gradient of a field that feeds several propagators). */
#define XL_ACCUMULATE 4

/* Sampling grid: x_m = x0 + m dx, y_n = y0 + n dy. */
typedef struct xl_grid {
  int32_t nx, ny;
  double dx, dy, x0, y0;
} xl_grid;

/* CZT output window: X_p = xo0 + p dxo (p < mx), Y_q = yo0 + q dyo (q < my). */
typedef struct xl_window {
  int32_t mx, my;
  double dxo, dyo, xo0, yo0;
} xl_window;

/* Library version string. */
const char* xl_version(void);

/* Message of the last failing call on this host thread ("" if none). */
const char* xl_last_error(void);

/* Frees every cached spectrum / chirp table and every workspace (synchronises the device). */
xl_status xl_cache_clear(void);

/* Bytes currently held by the spectrum cache and the workspaces. */
int64_t xl_cache_bytes(void);

/* Diagnostics (not part of the method). Number of kernels the library has launched since it was
 * loaded (a host-side counter incremented at every launch). */
int64_t xl_launch_count(void);

/* While on (on != 0), every launch is bracketed by CUDA events recorded on its own stream. */
xl_status xl_profile_enable(int32_t on);

/* Synchronises on the recorded events and writes one line "name launches total_ms" per kernel
 * family into buf (NUL-terminated, truncated to len), then clears the records. Returns the bytes
 * the full report needs. buf may be NULL to query the size (the records are still cleared). */
int32_t xl_profile_report(char* buf, int32_t len);

/* ---------------------------------------------------------------------------------------------
 * Scalar RS propagation (Methods, "Features and performance": FFT-based numerical integration of
 * the Rayleigh-Sommerfeld integral).
 *
 * Discrete definition (reading: first RS integral, rectangle rule, output grid = input grid):
 *   u_out[q][p] = sum_{n<ny, m<nx} u_in[n][m] h[p-m][q-n],
 *   h[a][b] = (dx dy / 2 pi) z (1/r - i k) exp(i k r) / r^2,  r = sqrt((a dx)^2 + (b dy)^2 + z^2).
 * Realisation: zero-pad to [2ny][2nx], 2D FFT, multiply by the cached 2D DFT of h placed at
 * (a mod 2nx, b mod 2ny), inverse FFT, crop.
 *
 * u_in, u_out: [batch][ny][nx] complex (dtype). u_out may not alias u_in.
 * z:           [batch] distances (> 0); host array, or device array with flags & XL_Z_DEVICE
 *              (then the transfer spectrum is regenerated in-stream on every call).
 * Supported:   nx, ny powers of two in [32, 4096]; batch >= 0 (0 is a no-op).
 * -------------------------------------------------------------------------------------------*/
xl_status xl_rs_propagate(const void* u_in, void* u_out, int32_t batch, const xl_grid* grid,
                          double wavelength, const double* z, int32_t flags, int32_t dtype,
                          void* stream);

/* Adjoint of xl_rs_propagate (same sizes):
 *   g_in = P^H g_out   (convolution with conj(h[-a][-b]), i.e. the spectrum conj(H)),
 *   g_z[b] = Re sum conj(g_out) dU_out/dz   (dh/dz spectrum, Parseval in the frequency domain).
 * g_in may be NULL (no field gradient); g_z may be NULL (no distance gradient) and needs u_in.
 * g_z: [batch] doubles, device memory, overwritten. */
xl_status xl_rs_propagate_backward(const void* g_out, const void* u_in, void* g_in, double* g_z,
                                   int32_t batch, const xl_grid* grid, double wavelength,
                                   const double* z, int32_t flags, int32_t dtype, void* stream);

/* Forward RS that also keeps what the adjoint's distance gradient needs from the input: the 2D
 * spectrum of the zero-padded input (the column transforms the convolution computes anyway), so
 * that xl_rs_propagate_backward_saved transforms nothing of the input again. The paper computes
 * the same gradient by reverse-mode differentiation (which keeps its forward intermediates in the
 * same way).
 *   saved: [batch][2 nx][2 ny] complex (dtype; row kx holds the spectrum's column kx), caller-owned
 *          device memory of batch * 4 * nx * ny * (8 or 16) bytes, overwritten; may not alias
 *          u_in or u_out.
 * Everything else as xl_rs_propagate (u_out is bit-identical to its result). */
xl_status xl_rs_propagate_save(const void* u_in, void* u_out, void* saved, int32_t batch,
                               const xl_grid* grid, double wavelength, const double* z,
                               int32_t flags, int32_t dtype, void* stream);

/* Adjoint of xl_rs_propagate taking the spectra saved by xl_rs_propagate_save (same grid,
 * wavelength, distances and dtype) in place of u_in; g_in is bit-identical to that of
 * xl_rs_propagate_backward, g_z equal to it up to rounding (its sum runs in another kernel).
 * saved may be NULL when g_z is NULL. */
xl_status xl_rs_propagate_backward_saved(const void* g_out, const void* saved, void* g_in,
                                         double* g_z, int32_t batch, const xl_grid* grid,
                                         double wavelength, const double* z, int32_t flags,
                                         int32_t dtype, void* stream);

/* Scalar RS propagation that allocates nothing. The paper has no counterpart: this entry point
 * serves callers that cannot let a library allocate device memory (memory owned by another
 * runtime's allocator, hosts that reserve all device memory up front, sandboxes without the
 * allocation API). It computes the discrete RS convolution of xl_rs_propagate, equal to it within
 * rounding (not bit for bit: other kernel variants, see xl_rs_static.cu), for complex64 fields
 * with nx, ny powers of two in [32, 256]; larger grids return XL_ERR_UNSUPPORTED. Its scratch
 * (twiddles, spectra, the transposed intermediate) is one fixed 2,136,320-byte static device array
 * that every GPU loading the library keeps until the process exits. No cudaMalloc / cudaFree is
 * called; the transfer spectrum is regenerated for every run of equal consecutive distances.
 *  - The first call on each device does a one-time set-up (looks up the array's device address
 *    and fills its twiddle tables, synchronising `stream`): make that first call before any
 *    stream capture.
 *  - Every call uses the same array: calls that overlap on the GPU (different streams, or
 *    threads without ordering) race and corrupt each other's results. Order them.
 *  - The set-up is kept for the life of the process: a cudaDeviceReset after the first call is
 *    not supported (the array's contents are lost with the context).
 * u_in, u_out: [batch][ny][nx] complex64 device arrays (not aliasing); z: host [batch] (> 0). */
xl_status xl_rs_propagate_static(const void* u_in, void* u_out, int32_t batch, const xl_grid* grid,
                                 double wavelength, const double* z, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Vectorial RS (Methods, "Features and performance"; VRS of Ye et al., cited with RS).
 * Reading: Ex' = h * Ex, Ey' = h * Ey, Ez' = h_x * Ex + h_y * Ey with
 *   h_x[a][b] = -(a dx / z) h[a][b],  h_y[a][b] = -(b dy / z) h[a][b]
 * (the divergence-free completion of the transverse RS field).
 * exy_in: [batch][2][ny][nx]; exyz_out: [batch][3][ny][nx]. Other arguments as xl_rs_propagate.
 * -------------------------------------------------------------------------------------------*/
xl_status xl_vrs_propagate(const void* exy_in, void* exyz_out, int32_t batch, const xl_grid* grid,
                           double wavelength, const double* z, int32_t flags, int32_t dtype,
                           void* stream);

/* Adjoint of xl_vrs_propagate: g_exyz [batch][3][ny][nx] -> g_exy [batch][2][ny][nx] (nullable),
 * g_z [batch] (nullable, needs exy_in). */
xl_status xl_vrs_propagate_backward(const void* g_exyz, const void* exy_in, void* g_exy,
                                    double* g_z, int32_t batch, const xl_grid* grid,
                                    double wavelength, const double* z, int32_t flags,
                                    int32_t dtype, void* stream);

/* VRS counterparts of xl_rs_propagate_save / xl_rs_propagate_backward_saved:
 * saved: [batch][2][2 nx][2 ny] complex (the spectra of Ex and Ey). */
xl_status xl_vrs_propagate_save(const void* exy_in, void* exyz_out, void* saved, int32_t batch,
                                const xl_grid* grid, double wavelength, const double* z,
                                int32_t flags, int32_t dtype, void* stream);
xl_status xl_vrs_propagate_backward_saved(const void* g_exyz, const void* saved, void* g_exy,
                                          double* g_z, int32_t batch, const xl_grid* grid,
                                          double wavelength, const double* z, int32_t flags,
                                          int32_t dtype, void* stream);


/* ---------------------------------------------------------------------------------------------
 * CZT propagation onto an output window (Methods, "Features and performance": the chirped
 * z-transform, an accelerated RS variant that samples an arbitrary region of interest; Bluestein
 * method of the cited Hu et al.).
 * Reading: the Fresnel form of the RS integral evaluated on the window,
 *   u_out[q][p] = exp(ikz)/(i lambda z) dx dy sum_{n,m} u_in[n][m]
 *                 exp(i k [(X_p - x_m)^2 + (Y_q - y_n)^2] / (2 z)),
 * realised by Bluestein chirp multiplies and padded FFT convolutions separately along x and y.
 * Each axis's grid side is cut into S segments whose transforms are summed before one inverse
 * transform (length L = 2^ceil(log2(ceil(N/S) + M - 1))); S is chosen per axis to minimise the
 * transform work (2048 -> 512: S = 4, L = 1024).
 * vectorial = 0: u_in [batch][ny][nx] -> u_out [batch][my][mx].
 * vectorial = 1: u_in [batch][2][ny][nx] (Ex, Ey) -> u_out [batch][3][my][mx] (Ex', Ey', Ez'),
 *   Ez' = sum [-(X_p - x_m)/z Ex - (Y_q - y_n)/z Ey] K (the VRS kernel ratio applied to CZT).
 * vectorial = 2: as 1, but u_in is a 3-component field [batch][3][ny][nx] whose Ez plane is not
 *   used (the propagated Ez follows from the transverse components); the adjoint writes a zero
 *   gradient into that plane.
 * Supported: any nx, ny, mx, my >= 1 with N + M - 1 <= 8192 per axis. z as in xl_rs_propagate.
 * -------------------------------------------------------------------------------------------*/
xl_status xl_czt_propagate(const void* u_in, void* u_out, int32_t batch, int32_t vectorial,
                           const xl_grid* grid, const xl_window* window, double wavelength,
                           const double* z, int32_t flags, int32_t dtype, void* stream);

/* Adjoint of xl_czt_propagate and its distance gradient:
 *   g_in = C^H g_out: g_out [batch][1 or 3][my][mx] -> g_in [batch][1, 2 or 3][ny][nx]
 *     (the conjugate-chirp convolutions in reverse order); g_in may be NULL.
 *   g_z[b] = Re sum conj(g_out) du_out/dz (device doubles, nullable; needs u_in, the forward's
 *     input), from dK/dz = K [ik - 1/z - ik ((X_p - x_m)^2 + (Y_q - y_n)^2) / (2 z^2)] (and, for
 *     vectorial fields, the z-dependence of the Ez kernel ratio). This call forms the forward's
 *     saved sums itself (the cost of one forward with them); xl_czt_propagate_backward_saved
 *     reads those of an earlier xl_czt_propagate_save instead.
 * flags: XL_Z_DEVICE; XL_PHASE_INVARIANT (the loss is blind to a constant phase on u_out) drops
 * the Re(ik <g_out, u_out>) term of g_z; XL_ACCUMULATE adds to g_in and g_z (the Ez plane of a
 * 3-component g_in is then left as it is). */
xl_status xl_czt_propagate_backward(const void* g_out, const void* u_in, void* g_in, double* g_z,
                                    int32_t batch, int32_t vectorial, const xl_grid* grid,
                                    const xl_window* window, double wavelength, const double* z,
                                    int32_t flags, int32_t dtype, void* stream);

/* Complex elements (of dtype) per batch element of the buffer xl_czt_propagate_save fills: the
 * x-pass intermediate, the forward's distance-gradient sums along x and y and the per-component
 * window fields. -1 for unsupported sizes. The layout depends on the sizes, vectorial and dtype
 * only. */
int64_t xl_czt_save_elems(const xl_grid* grid, const xl_window* window, int32_t vectorial,
                          int32_t dtype);

/* Forward CZT that also writes, into the caller's `saved` buffer ([batch][xl_czt_save_elems]
 * complex elements, device), what the adjoint's distance gradient needs from the forward, so that
 * xl_czt_propagate_backward_saved transforms nothing of the input again. u_out as
 * xl_czt_propagate. saved may not alias u_in or u_out. */
xl_status xl_czt_propagate_save(const void* u_in, void* u_out, void* saved, int32_t batch,
                                int32_t vectorial, const xl_grid* grid, const xl_window* window,
                                double wavelength, const double* z, int32_t flags, int32_t dtype,
                                void* stream);

/* xl_czt_propagate_backward with the sums an earlier xl_czt_propagate_save (same sizes, distances
 * and dtype) left in `saved`; u_in (its input) is still read for g_z. saved may be NULL when g_z
 * is NULL. */
xl_status xl_czt_propagate_backward_saved(const void* g_out, const void* u_in, const void* saved,
                                          void* g_in, double* g_z, int32_t batch, int32_t vectorial,
                                          const xl_grid* grid, const xl_window* window,
                                          double wavelength, const double* z, int32_t flags,
                                          int32_t dtype, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Angular-spectrum CZT: the exact-RS reading of the CZT propagator (Methods, "Features and
 * performance": propagation onto an arbitrarily placed and sampled window; the CZT of Hu et al.
 * evaluates the inverse transform of the propagated angular spectrum on the window).
 * Reading: with signed DFT frequencies f = j / (nx dx), g = l / (ny dy), j, l in [-n/2, n/2),
 *   U^(f, g) = sum_{n,m} u_in[n][m] exp(-2 pi i (f x_m + g y_n)),
 *   u_out[q][p] = 1/(nx ny) sum_{f,g} U^(f, g) exp(i z kz) exp(2 pi i (f X_p + g Y_q)),
 *   kz = sqrt(k^2 - (2 pi f)^2 - (2 pi g)^2) (kz = i sqrt(...) beyond the light cone: decay).
 * On the native grid (window = grid) this is the angular-spectrum method; there is no paraxial
 * approximation. Realised by two spectrum passes (the field times (-1)^(x+y), row and column
 * transforms, the transfer function cached per distance) and the two Bluestein window passes.
 * u_in: [batch][ny][nx], u_out: [batch][my][mx] (complex dtype, device, not aliasing).
 * z: [batch] distances >= 0 (host, or device with XL_Z_DEVICE).
 * Supported: nx, ny powers of two in [64, 4096]; mx, my >= 1 with N + M - 1 <= 8192 per axis.
 * -------------------------------------------------------------------------------------------*/
xl_status xl_asczt_propagate(const void* u_in, void* u_out, int32_t batch, const xl_grid* grid,
                             const xl_window* window, double wavelength, const double* z,
                             int32_t flags, int32_t dtype, void* stream);

/* Adjoint of xl_asczt_propagate: g_out [batch][my][mx] -> g_in [batch][ny][nx] (nullable) and
 * g_z[b] = Re sum conj(g_out) du_out/dz (device doubles, nullable; needs u_in), the distance
 * derivative of the transfer function being i kz exp(i z kz). */
xl_status xl_asczt_propagate_backward(const void* g_out, const void* u_in, void* g_in,
                                      double* g_z, int32_t batch, const xl_grid* grid,
                                      const xl_window* window, double wavelength, const double* z,
                                      int32_t flags, int32_t dtype, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Optical elements (Methods, "Features and performance": SLMs (one free phase per pixel), the
 * super-SLM (independent phases on the horizontal and vertical components), polarisers, variable
 * retarders / wave plates, planar lenses). A chain of up to 8 elements is applied in one pass.
 * Readings (the paper names the elements only):
 *   XL_SLM        every component times exp(i phi_x)
 *   XL_SSLM       Ex times exp(i phi_x), Ey times exp(i phi_y)
 *   XL_LENS       every component times exp(-i k (x^2 + y^2) / (2 f))
 *   XL_POLARIZER  J = R(-alpha) diag(1, 0) R(alpha)
 *   XL_WAVEPLATE  J = R(-theta) diag(1, exp(i eta)) R(theta), R(t) = [[cos t, sin t], [-sin t, cos t]]
 *                 (a half-wave plate is eta = pi)
 *   XL_TO_VECTOR  (Ex, Ey) = (u, 0): an x-polarised scalar field becomes a 2-component field
 * -------------------------------------------------------------------------------------------*/
#define XL_SLM 0
#define XL_SSLM 1
#define XL_LENS 2
#define XL_POLARIZER 3
#define XL_WAVEPLATE 4
#define XL_TO_VECTOR 5

typedef struct xl_element {
  int32_t kind;
  int32_t reserved;
  const void* phi_x;   /* device phase mask(s) [ny][nx] (float for XL_C64, double for XL_C128) */
  const void* phi_y;   /* second mask of XL_SSLM */
  int64_t phi_stride;  /* elements between the masks of consecutive batch entries; 0 = shared */
  double f, alpha, eta, theta; /* host parameters (used unless flags & XL_Z_DEVICE) */
} xl_element;

/* in: [batch][comps_in][ny][nx] (comps_in 1, 2 or 3); out: [batch][comps_out][ny][nx] where
 * comps_out = 2 if the chain contains XL_TO_VECTOR, else comps_in. For 3-component fields
 * (Ex, Ey, Ez) masks and lenses act on all components, Jones elements on (Ex, Ey) only. out may
 * alias in when comps_out == comps_in.
 * params: with flags & XL_Z_DEVICE, device doubles [batch][n_elem][4] = {f, alpha, eta, theta}
 * replacing the host values of every element (for parameters trained on the device); else NULL. */
xl_status xl_apply_elements(const void* in, void* out, int32_t batch, int32_t comps_in,
                            const xl_grid* grid, double wavelength, const xl_element* elements,
                            int32_t n_elem, const double* params, int32_t flags, int32_t dtype,
                            void* stream);

/* Adjoint of xl_apply_elements at the forward input `in`:
 *   g_in = J^H g_out element by element in reverse (NULL: not written);
 *   g_phi_x[e], g_phi_y[e]: dL/dphi = Im(g_out conj(u_out)) per pixel, laid out like the masks;
 *     a shared mask (phi_stride 0) receives the sum over the batch (arrays and entries nullable);
 *   g_params: device [batch][n_elem][4] dL/d{f, alpha, eta, theta} (nullable).
 * Shared and per-batch masks may not both request gradients in one call (XL_ERR_UNSUPPORTED). */
xl_status xl_apply_elements_backward(const void* g_out, const void* in, void* g_in, int32_t batch,
                                     int32_t comps_in, const xl_grid* grid, double wavelength,
                                     const xl_element* elements, int32_t n_elem,
                                     const double* params, int32_t flags, void* const* g_phi_x,
                                     void* const* g_phi_y, double* g_params, int32_t dtype,
                                     void* stream);

/* ---------------------------------------------------------------------------------------------
 * Camera intensity and losses (Methods, "Loss function"; camera intensities |Ex|^2 + |Ey|^2,
 * |Ez|^2 or total as in the Results).
 *   I = sum over the components selected by comp_mask (bit c = component c) of |E_c|^2.
 *   XL_SECOND_MOMENT (reading; the paper's spot metric is (pi/4) FWHMx FWHMy):
 *       L = sum I ((x - xbar)^2 + (y - ybar)^2) / sum I, xbar = sum I x / sum I (grid units^2).
 *   XL_DENSITY: L = Area / I_eps, I_eps = sum of I over pixels with I > eps * max(I) (strict),
 *       Area = their count.
 * field: [batch][comps][ny][nx]; loss: device doubles [batch]; intensity: nullable device
 * [batch][ny][nx] (float for XL_C64, double for XL_C128). A non-finite loss is reported by
 * xl_device_status().
 * -------------------------------------------------------------------------------------------*/
#define XL_SECOND_MOMENT 0
#define XL_DENSITY 1
#define XL_MSE 2 /* mean (I - I_target)^2 (Results, "Data-driven rediscovery"); needs the _ex form */

xl_status xl_intensity_loss(const void* field, int32_t batch, int32_t comps, uint32_t comp_mask,
                            const xl_grid* grid, int32_t mode, double eps, double* loss,
                            void* intensity, int32_t dtype, void* stream);

/* g_field = 2 g_loss[b] dL/dI E on the selected components, 0 on the others.
 *   second moment: dL/dI = [(x - xbar)^2 + (y - ybar)^2 - L] / sum I
 *   density:       dL/dI = -Area / I_eps^2 above the threshold, 0 elsewhere
 * g_loss: device doubles [batch] or NULL (= 1). g_field: [batch][comps][ny][nx], not aliasing. */
xl_status xl_intensity_loss_backward(const void* field, int32_t batch, int32_t comps,
                                     uint32_t comp_mask, const xl_grid* grid, int32_t mode,
                                     double eps, const double* g_loss, void* g_field,
                                     int32_t dtype, void* stream);

/* Extended camera losses.
 *   field_dep (nullable): a depletion field of the same layout; I is then the STED effective
 *     intensity (Methods, "Stimulated emission depletion model")
 *       I_eff = I_ex [1 - beta (1 - exp(-I_dep / I_ex))], I_eff = 0 where I_ex = 0,
 *     with I_ex, I_dep the selected-component intensities of field and field_dep, 0 <= beta <= 1.
 *   target (XL_MSE only): device [batch][ny][nx] target intensities (float / double).
 * Other arguments as xl_intensity_loss. */
xl_status xl_intensity_loss_ex(const void* field, const void* field_dep, const void* target,
                               int32_t batch, int32_t comps, uint32_t comp_mask,
                               const xl_grid* grid, int32_t mode, double eps, double beta,
                               double* loss, void* intensity, int32_t dtype, void* stream);

/* Gradient of xl_intensity_loss_ex: g_field (and g_field_dep when field_dep is given) through
 *   dI_eff/dI_ex = 1 - beta + beta e^{-r} (1 + r),  dI_eff/dI_dep = -beta e^{-r},  r = I_dep/I_ex
 * (limits (1 - beta, 0) at I_ex = 0); XL_MSE: dL/dI = 2 (I - I_target) / (nx ny). */
xl_status xl_intensity_loss_ex_backward(const void* field, const void* field_dep,
                                        const void* target, int32_t batch, int32_t comps,
                                        uint32_t comp_mask, const xl_grid* grid, int32_t mode,
                                        double eps, double beta, const double* g_loss,
                                        void* g_field, void* g_field_dep, int32_t dtype,
                                        void* stream);

/* The loss and its field gradient in one call (an optimiser step needs both): loss[b] as
 * xl_intensity_loss_ex and g_field (g_field_dep) as xl_intensity_loss_ex_backward with
 * g_loss = 1, from one set of the statistics sweeps (three passes over the field instead of
 * five for the two calls). Arguments and errors as those two. */
xl_status xl_intensity_loss_and_grad(const void* field, const void* field_dep, const void* target,
                                     int32_t batch, int32_t comps, uint32_t comp_mask,
                                     const xl_grid* grid, int32_t mode, double eps, double beta,
                                     double* loss, void* g_field, void* g_field_dep, int32_t dtype,
                                     void* stream);

/* Softmin over detectors (Methods, "Rediscovery through exploration of optical topologies": the
 * parameter update follows the detector with the smallest loss through a smooth minimum):
 *   out[b] = -log(sum_d exp(-beta losses[b][d])) / beta,
 *   weights[b][d] = d out[b] / d losses[b][d] (nullable). Device doubles; beta > 0. */
xl_status xl_softmin(const double* losses, int32_t batch, int32_t n_det, double beta, double* out,
                     double* weights, void* stream);

/* Synchronises `stream`, then returns and clears the device status: XL_ERR_NONFINITE if a loss
 * reduction produced a non-finite value since the last call, XL_ERR_TIMEOUT if a kernel gave up
 * waiting for a bulk tensor copy (a bounded wait), else XL_OK. After XL_ERR_TIMEOUT every output
 * of that launch and of every later launch is undefined, not only the rows that were skipped: a
 * block that gave up may still have copies in flight into shared memory that a later block is
 * given. */
xl_status xl_device_status(void* stream);

/* ---------------------------------------------------------------------------------------------
 * Autotuner of the transposing row passes (the batch scheduler's launch plan; the paper has no
 * counterpart: its JAX/XLA back end picks launch shapes itself). Families (XL_TUNE_*): RS passes
 * 1 and 3 and the four CZT window passes; variants: 0 the built-in rows per block, 1 half as
 * many, 2 twice as many where a block stays within 1024 threads and an SM's shared memory; these
 * give bit-identical results (rows shorter than 1024 always use variant 0). The complex64 scalar
 * CZT passes of lengths 512, 1024 and 2048 have two more: the built-in rows with FFT radix plan 1
 * (3) or plan 2 (4), the transform's radix-2/4/8 stage first or second instead of last (equal
 * results within rounding). Choices are process-wide (host memory).
 * -------------------------------------------------------------------------------------------*/
#define XL_TUNE_RS_PASS1 0
#define XL_TUNE_RS_PASS3 1
#define XL_TUNE_CZT_FWD_X 2
#define XL_TUNE_CZT_FWD_Y 3
#define XL_TUNE_CZT_ADJ_X 4
#define XL_TUNE_CZT_ADJ_Y 5

/* Times every variant of the passes a grid (and, when window is non-NULL, a CZT onto that
 * window) uses, `reps` launches each on `stream` with synthetic data (allocates and frees its own
 * device buffers, synchronises `stream`), and keeps the fastest. Each timed launch processes
 * enough planes (up to 16) that its data exceeds L2, as batched calls do. */
xl_status xl_autotune(const xl_grid* grid, const xl_window* window, int32_t dtype, int32_t reps,
                      void* stream);
/* The variant used for (family, row length L, dtype): 0..4, or -1 for an unknown family. */
int32_t xl_tune_get(int32_t family, int32_t L, int32_t dtype);
/* Sets a variant by hand (XL_ERR_ARG for an unknown family, L, dtype or variant). */
xl_status xl_tune_set(int32_t family, int32_t L, int32_t dtype, int32_t variant);
xl_status xl_tune_clear(void);
/* Text file of the choices, one "family L dtype variant microseconds" line each. Loading a
 * malformed file returns XL_ERR_ARG and applies nothing. */
xl_status xl_tune_save(const char* path);
xl_status xl_tune_load(const char* path);

/* ---------------------------------------------------------------------------------------------
 * Beam splitters (Results, "Towards large-scale discovery"; Methods, "The large-scale search
 * space": beam splitters with a continuous ratio in [0, 1] connect the paths of the table).
 * Reading: lossless and non-polarising, R = reflected intensity fraction, t = sqrt(1 - R),
 * r = sqrt(R), the reflected amplitude carrying the factor i:
 *   out_t = t a + i r b,   out_r = i r a + t b    (every component alike).
 * a, b, out_t, out_r: [batch][elems] complex (dtype) device arrays, `elems` = components x pixels
 *   of one batch element; a or b NULL is a zero input, out_t or out_r NULL is not written.
 *   Outputs may alias inputs (each element is read before it is written).
 * R: [batch] device doubles in [0, 1] (trainable).
 * Errors: XL_ERR_ARG for a NULL R (non-empty call), negative sizes or a bad dtype;
 *   XL_ERR_UNSUPPORTED for batch > 65535.
 * -------------------------------------------------------------------------------------------*/
xl_status xl_beam_splitter(const void* a, const void* b, void* out_t, void* out_r, int32_t batch,
                           int64_t elems, const double* R, int32_t dtype, void* stream);

/* Adjoint: g_a = t g_t - i r g_r, g_b = -i r g_t + t g_r (each nullable), and
 * g_R[b] = dL/dR = Re sum conj(g_t) d out_t/dR + conj(g_r) d out_r/dR (device doubles,
 * nullable; needs the forward inputs a, b). dL/dR is unbounded at R = 0 and R = 1 (inf or NaN
 * there): optimise an unconstrained parameter mapped into (0, 1). g_t, g_r NULL: zero. */
xl_status xl_beam_splitter_backward(const void* g_t, const void* g_r, const void* a, const void* b,
                                    void* g_a, void* g_b, double* g_R, int32_t batch, int64_t elems,
                                    const double* R, int32_t dtype, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Adam (the paper's optimiser): bias-corrected step t >= 1,
 *   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;  p -= lr m/(1-b1^t) / (sqrt(v/(1-b2^t)) + eps).
 * params, m, v, grad: device arrays of n reals (real_dtype 0 = float, 1 = double), updated in
 * place. t is read from t_dev (device int32, for graph replay) when non-NULL, else t_host.
 * -------------------------------------------------------------------------------------------*/
xl_status xl_adam_step(void* params, void* m, void* v, const void* grad, int64_t n,
                       int32_t real_dtype, double lr, double beta1, double beta2, double eps,
                       const int32_t* t_dev, int32_t t_host, void* stream);

/* AdamW (decoupled weight decay, used by the paper's data-driven and topology runs with
 * weight decay 1e-4): the Adam step above and p -= lr * weight_decay * p (p before the step). */
xl_status xl_adamw_step(void* params, void* m, void* v, const void* grad, int64_t n,
                        int32_t real_dtype, double lr, double beta1, double beta2, double eps,
                        double weight_decay, const int32_t* t_dev, int32_t t_host, void* stream);

/* *t_dev += 1 in stream order. */
xl_status xl_step_advance(int32_t* t_dev, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Batched optical-table optimisation (the paper batches independent setups / samples with vmap:
 * Methods "Data-driven rediscovery", "Features and performance"; virtual tables of Results
 * "Towards large-scale discovery"). Every setup is the table
 *   x-polarised Gaussian -> SLM1 (phi1) -> RS z1 -> SLM2 (phi2) -> to-vector -> half-wave plate
 *   (theta) -> VRS z2 -> lens f -> VCZT f onto the camera -> second-moment spot size of the
 *   total intensity,
 * with its own grid size N (pitch = extent / N), masks, theta, z1 and z2. Setups are grouped by N
 * and each stage of a group runs as one batched library call with device-resident parameters.
 * xl_batch_step runs forward, backward and one Adam step (lr for masks and theta, lr_z for the
 * distances; beta1 0.9, beta2 0.999, eps 1e-8) for all setups. With use_graph the step runs on a
 * stream owned by the batch, ordered after and before `stream` by events: the first such call is
 * eager (it sizes every workspace), the second captures the step into a CUDA graph, and every
 * later call replays that graph.
 * Masks start uniform in [0, 2 pi): SplitMix64 (seed + setup index for phi1, + 0x10000 for phi2),
 * one draw per pixel in row-major order; the source is exp(-rho^2 / w0^2).
 * -------------------------------------------------------------------------------------------*/
typedef struct xl_table_config {
  double wavelength; /* lambda */
  double extent;     /* physical width of every input grid (pitch = extent / N) */
  double w0;         /* source waist */
  double f;          /* lens focal length = VCZT distance */
  double cam_width;  /* camera window width (centred) */
  double lr;         /* Adam step size for the masks and theta */
  double lr_z;       /* Adam step size for z1 and z2 */
  int32_t cam_m;     /* camera pixels per side */
  int32_t dtype;     /* XL_C64 or XL_C128 */
  int32_t checkpoint; /* what the RS / VRS adjoints read for their distance gradients (per-plane
                         checkpointing): 0 = the 2D spectra of their zero-padded inputs, kept by
                         the forwards (12 field planes a setup, no input transform in the
                         adjoints); 1 = only the fields at the optical planes, the adjoints
                         transforming their inputs again (about half the memory a setup);
                         XL_CHECKPOINT_AUTO = 0 when the batch fits in memory_budget, else 1. */
  int64_t memory_budget; /* 0 = no limit; else the most device memory the batch's own buffers may
                            hold (the figure xl_batch_memory reports): xl_batch_create returns
                            XL_ERR_NOMEM, allocating nothing, when the resolved mode needs more */
} xl_table_config;

#define XL_CHECKPOINT_AUTO 2

typedef struct xl_batch xl_batch; /* opaque; owns all per-setup device buffers */

/* grid_n: [n_setups] powers of two in [32, 4096]; init: host [n_setups][3] = {theta, z1, z2}.
 * Allocates with cudaMalloc (call outside stream capture). */
xl_status xl_batch_create(const xl_table_config* cfg, int32_t n_setups, const int32_t* grid_n,
                          const double* init, uint64_t seed, xl_batch** out, void* stream);

/* Device bytes xl_batch_create allocates for these setups (what xl_batch_memory then reports) in
 * the checkpoint mode cfg->checkpoint resolves to; that mode (0 or 1) goes to *mode_out
 * (nullable). -1 for a NULL or invalid argument. Host arithmetic only: no device call. */
int64_t xl_batch_plan_memory(const xl_table_config* cfg, int32_t n_setups, const int32_t* grid_n,
                             int32_t* mode_out);

/* One optimisation step of every setup (see above). */
xl_status xl_batch_step(xl_batch* batch, int32_t use_graph, void* stream);

#define XL_BATCH_LOSS 0         /* double: the loss of the last step (before its Adam update) */
#define XL_BATCH_SCALARS 1      /* double[3]: theta, z1, z2 (current values) */
#define XL_BATCH_GRAD_SCALARS 2 /* double[3]: dL/dtheta, dL/dz1, dL/dz2 of the last step */
#define XL_BATCH_PHI1 3         /* real[N][N] (float for XL_C64, double for XL_C128) */
#define XL_BATCH_PHI2 4
#define XL_BATCH_GRAD_PHI1 5
#define XL_BATCH_GRAD_PHI2 6

/* Device bytes the batch's own buffers hold (fields, gradients, masks, moments, parameters; the
 * library's shared workspaces and table cache are reported by xl_cache_bytes). -1 for NULL. */
int64_t xl_batch_memory(xl_batch* batch);

/* Copies one quantity of one setup to host memory (synchronises the stream). */
xl_status xl_batch_read(xl_batch* batch, int32_t what, int32_t setup, void* host_out, void* stream);

/* Grid size N of a setup (-1 if out of range). */
int32_t xl_batch_grid(xl_batch* batch, int32_t setup);

/* Frees every buffer and the captured graph (synchronises the device). */
xl_status xl_batch_destroy(xl_batch* batch);

#ifdef __cplusplus
}
#endif

#endif /* XL_H_ */
