// FP64 CPU oracle for free-space propagation, optical elements and camera losses.
//
// TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU-baseline leg of the
// benchmark may load this library. It shares no code, header, table or helper with the CUDA
// path: every formula here is written out again from the paper's description of the method
// and from the discrete readings listed at each function.
//
// Paper: XLuminA (arXiv 2310.08408), Methods, "Features and performance": light is propagated
// by FFT-based numerical integration of the Rayleigh-Sommerfeld integral (RS), its vectorial
// form (VRS), and the chirped z-transform (CZT / VCZT) onto an arbitrary output window.
// The paper prints no formula for these; the discrete definitions below are the readings
// stated at each function (rectangle rule, same output grid, zero-padding to 2N).
//
// Conventions (readings): time dependence exp(-i w t), outgoing waves exp(+i k r);
// k = 2 pi / lambda; grids x_m = x0 + m dx; complex data interleaved (re, im), row-major
// [ny][nx] with x fastest; gradients g = dL/dRe u + i dL/dIm u.
//
// Arithmetic is plain double precision with std::complex<double>; the FFT is a textbook
// radix-2 Cooley-Tukey transform with every twiddle evaluated directly by cos/sin.

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <functional>
#include <thread>
#include <vector>

typedef std::complex<double> cd;
static const double PI = 3.14159265358979323846264338327950288;

static int g_threads = 0;

static int n_threads() {
  int t = g_threads > 0 ? g_threads : (int)std::thread::hardware_concurrency();
  return t < 1 ? 1 : t;
}

// Runs fn(begin, end) over [0, n) split into contiguous chunks, one per thread.
static void parallel_for(int64_t n, const std::function<void(int64_t, int64_t)>& fn) {
  int64_t T = std::min<int64_t>(n_threads(), n);
  if (T <= 1) {
    fn(0, n);
    return;
  }
  std::vector<std::thread> pool;
  for (int64_t t = 0; t < T; ++t) pool.emplace_back(fn, n * t / T, n * (t + 1) / T);
  for (auto& th : pool) th.join();
}

static inline cd ld(const double* p, int64_t i) { return cd(p[2 * i], p[2 * i + 1]); }
static inline void st(double* p, int64_t i, cd v) {
  p[2 * i] = v.real();
  p[2 * i + 1] = v.imag();
}

static bool is_pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }

// ------------------------------------------------------------------------------------------
// FFT: unnormalised DFT X[k] = sum_j x[j] exp(sign * 2 pi i j k / n), n a power of two.
// Iterative radix-2 Cooley-Tukey (bit-reversal permutation, then log2 n butterfly sweeps).
// ------------------------------------------------------------------------------------------
static void fft_inplace(cd* x, int64_t n, int sign) {
  for (int64_t i = 1, j = 0; i < n; ++i) {
    int64_t bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(x[i], x[j]);
  }
  for (int64_t len = 2; len <= n; len <<= 1) {
    int64_t half = len / 2;
    for (int64_t k = 0; k < half; ++k) {
      double ang = sign * 2.0 * PI * (double)k / (double)len;
      cd w(std::cos(ang), std::sin(ang));
      for (int64_t s = 0; s < n; s += len) {
        cd a = x[s + k], b = x[s + k + half] * w;
        x[s + k] = a + b;
        x[s + k + half] = a - b;
      }
    }
  }
}

// 2D transform of a row-major [ny][nx] array: all rows, then all columns.
static void fft2_inplace(std::vector<cd>& a, int64_t ny, int64_t nx, int sign) {
  parallel_for(ny, [&](int64_t b, int64_t e) {
    for (int64_t r = b; r < e; ++r) fft_inplace(&a[r * nx], nx, sign);
  });
  parallel_for(nx, [&](int64_t b, int64_t e) {
    std::vector<cd> col(ny);
    for (int64_t c = b; c < e; ++c) {
      for (int64_t r = 0; r < ny; ++r) col[r] = a[r * nx + c];
      fft_inplace(col.data(), ny, sign);
      for (int64_t r = 0; r < ny; ++r) a[r * nx + c] = col[r];
    }
  });
}

// ------------------------------------------------------------------------------------------
// Rayleigh-Sommerfeld impulse responses (Methods, "Features and performance"; RS of the
// first kind as in the cited Shen & Wang FFT-DI method).
//
// Reading: the first RS integral U(x,y,z) = -(1/2pi) Int U0 d/dz[exp(ikr)/r] dA evaluated on
// an output grid equal to the input grid with a rectangle rule, so the discrete impulse
// response for pixel offset (a, b) is
//     h[a,b] = (dx dy / 2pi) z (1/r - i k) exp(i k r) / r^2,   r = sqrt((a dx)^2+(b dy)^2+z^2).
// Vectorial RS (Ye et al., cited with RS): the transverse components propagate with h, and
// the longitudinal one is Ez' = sum (Ex h_x + Ey h_y) with
//     h_x = -(a dx / z) h,   h_y = -(b dy / z) h,
// the choice that makes the propagated field divergence-free.
// The z-derivatives (used for distance gradients) follow by differentiating these:
//     dh/dz = (dx dy/2pi) exp(ikr) [ (1/r^3 - ik/r^2) + z^2 (k^2/r^3 + 3ik/r^4 - 3/r^5) ],
//     dh_x/dz = -(a dx/z) (dh/dz - h/z),  likewise for h_y.
// kind: 0 h, 1 h_x, 2 h_y, 3 dh/dz, 4 dh_x/dz, 5 dh_y/dz.
// ------------------------------------------------------------------------------------------
static cd rs_kernel(int kind, int64_t a, int64_t b, double dx, double dy, double z, double k) {
  double X = (double)a * dx, Y = (double)b * dy;
  double r = std::sqrt(X * X + Y * Y + z * z);
  double C = dx * dy / (2.0 * PI);
  cd I(0.0, 1.0);
  cd e = std::exp(I * (k * r));
  cd h = C * z * (1.0 / r - I * k) * e / (r * r);
  if (kind == 0) return h;
  if (kind == 1) return -(X / z) * h;
  if (kind == 2) return -(Y / z) * h;
  cd dh = C * e *
          ((1.0 / (r * r * r) - I * k / (r * r)) +
           z * z * (k * k / (r * r * r) + 3.0 * I * k / (r * r * r * r) - 3.0 / (r * r * r * r * r)));
  if (kind == 3) return dh;
  if (kind == 4) return -(X / z) * (dh - h / z);
  if (kind == 5) return -(Y / z) * (dh - h / z);
  return cd(0.0, 0.0);
}

// Kernel value used by a (possibly adjoint) convolution: the adjoint of convolution with k is
// convolution with conj(k[-a,-b]).
static cd conv_kernel(int kind, int adjoint, int64_t a, int64_t b, double dx, double dy, double z,
                      double k) {
  if (!adjoint) return rs_kernel(kind, a, b, dx, dy, z, k);
  return std::conj(rs_kernel(kind, -a, -b, dx, dy, z, k));
}

extern "C" {

void orc_set_threads(int n) { g_threads = n; }
int orc_get_threads(void) { return n_threads(); }

// In-place unnormalised 1D FFT of n complex values (n a power of two). Returns 0 or -1.
int orc_fft(double* x, int64_t n, int sign) {
  if (!is_pow2(n)) return -1;
  std::vector<cd> a(n);
  for (int64_t i = 0; i < n; ++i) a[i] = ld(x, i);
  fft_inplace(a.data(), n, sign);
  for (int64_t i = 0; i < n; ++i) st(x, i, a[i]);
  return 0;
}

// In-place unnormalised 2D FFT of a row-major [ny][nx] array.
int orc_fft2(double* x, int64_t ny, int64_t nx, int sign) {
  if (!is_pow2(nx) || !is_pow2(ny)) return -1;
  std::vector<cd> a(nx * ny);
  for (int64_t i = 0; i < nx * ny; ++i) a[i] = ld(x, i);
  fft2_inplace(a, ny, nx, sign);
  for (int64_t i = 0; i < nx * ny; ++i) st(x, i, a[i]);
  return 0;
}

// Direct O(n^2) DFT, any n: y[k] = sum_j x[j] exp(sign 2 pi i j k / n).
void orc_dft(const double* x, double* y, int64_t n, int sign) {
  for (int64_t kk = 0; kk < n; ++kk) {
    cd s(0.0, 0.0);
    for (int64_t j = 0; j < n; ++j) {
      double ang = sign * 2.0 * PI * (double)((j * kk) % n) / (double)n;
      s += ld(x, j) * cd(std::cos(ang), std::sin(ang));
    }
    st(y, kk, s);
  }
}

// Samples the impulse response of `kind` on offsets a in (-nx, nx), b in (-ny, ny) into a
// [(2ny-1)][(2nx-1)] table (index (b+ny-1, a+nx-1)).
void orc_rs_kernel_table(int kind, int64_t nx, int64_t ny, double dx, double dy, double wavelength,
                         double z, double* out) {
  double k = 2.0 * PI / wavelength;
  int64_t W = 2 * nx - 1;
  for (int64_t b = -(ny - 1); b <= ny - 1; ++b)
    for (int64_t a = -(nx - 1); a <= nx - 1; ++a)
      st(out, (b + ny - 1) * W + (a + nx - 1), rs_kernel(kind, a, b, dx, dy, z, k));
}

// RS convolution by zero-padded FFT (Methods: "FFT-based numerical integration of the RS
// integral"): pad the field to [2ny][2nx], place the sampled kernel at (a mod 2nx, b mod 2ny)
// for |a| < nx, |b| < ny (offset +-n itself is left 0), multiply the two 2D DFTs, inverse
// transform, divide by (2nx)(2ny), and keep [0,ny) x [0,nx). In exact arithmetic this is the
// linear convolution u_out[q][p] = sum_{n,m} u_in[n][m] K[p-m, q-n].
// adjoint != 0 applies the adjoint operator (kernel conj(K[-a,-b])).
int orc_rs_fft(const double* u_in, double* u_out, int64_t nx, int64_t ny, double dx, double dy,
               double wavelength, double z, int kind, int adjoint) {
  if (!is_pow2(nx) || !is_pow2(ny) || z <= 0.0) return -1;
  double k = 2.0 * PI / wavelength;
  int64_t Lx = 2 * nx, Ly = 2 * ny;
  std::vector<cd> hp(Lx * Ly, cd(0.0, 0.0)), up(Lx * Ly, cd(0.0, 0.0));
  parallel_for(2 * ny - 1, [&](int64_t bb, int64_t be) {
    for (int64_t t = bb; t < be; ++t) {
      int64_t b = t - (ny - 1);
      int64_t row = ((b % Ly) + Ly) % Ly;
      for (int64_t a = -(nx - 1); a <= nx - 1; ++a) {
        int64_t col = ((a % Lx) + Lx) % Lx;
        hp[row * Lx + col] = conv_kernel(kind, adjoint, a, b, dx, dy, z, k);
      }
    }
  });
  for (int64_t n = 0; n < ny; ++n)
    for (int64_t m = 0; m < nx; ++m) up[n * Lx + m] = ld(u_in, n * nx + m);
  fft2_inplace(hp, Ly, Lx, -1);
  fft2_inplace(up, Ly, Lx, -1);
  for (int64_t i = 0; i < Lx * Ly; ++i) up[i] *= hp[i];
  fft2_inplace(up, Ly, Lx, +1);
  double s = 1.0 / ((double)Lx * (double)Ly);
  for (int64_t n = 0; n < ny; ++n)
    for (int64_t m = 0; m < nx; ++m) st(u_out, n * nx + m, up[n * Lx + m] * s);
  return 0;
}

// The same convolution as a brute-force O(nx^2 ny^2) direct sum (the plain definition).
int orc_rs_direct(const double* u_in, double* u_out, int64_t nx, int64_t ny, double dx, double dy,
                  double wavelength, double z, int kind, int adjoint) {
  if (nx < 1 || ny < 1 || z <= 0.0) return -1;
  double k = 2.0 * PI / wavelength;
  int64_t W = 2 * nx - 1;
  std::vector<cd> tab(W * (2 * ny - 1));
  for (int64_t b = -(ny - 1); b <= ny - 1; ++b)
    for (int64_t a = -(nx - 1); a <= nx - 1; ++a)
      tab[(b + ny - 1) * W + (a + nx - 1)] = conv_kernel(kind, adjoint, a, b, dx, dy, z, k);
  std::vector<cd> u(nx * ny);
  for (int64_t i = 0; i < nx * ny; ++i) u[i] = ld(u_in, i);
  parallel_for(ny, [&](int64_t qb, int64_t qe) {
    for (int64_t q = qb; q < qe; ++q)
      for (int64_t p = 0; p < nx; ++p) {
        cd s(0.0, 0.0);
        for (int64_t n = 0; n < ny; ++n) {
          const cd* trow = &tab[(q - n + ny - 1) * W + (p + nx - 1)];
          const cd* urow = &u[n * nx];
          for (int64_t m = 0; m < nx; ++m) s += urow[m] * trow[-m];
        }
        st(u_out, q * nx + p, s);
      }
  });
  return 0;
}

// Direct sum at selected output pixels only: pts holds npts (p, q) pairs; out gets npts values.
int orc_rs_direct_points(const double* u_in, int64_t nx, int64_t ny, double dx, double dy,
                         double wavelength, double z, int kind, int adjoint, const int32_t* pts,
                         int64_t npts, double* out) {
  if (nx < 1 || ny < 1 || z <= 0.0) return -1;
  double k = 2.0 * PI / wavelength;
  parallel_for(npts, [&](int64_t ib, int64_t ie) {
    for (int64_t i = ib; i < ie; ++i) {
      int64_t p = pts[2 * i], q = pts[2 * i + 1];
      cd s(0.0, 0.0);
      for (int64_t n = 0; n < ny; ++n)
        for (int64_t m = 0; m < nx; ++m)
          s += ld(u_in, n * nx + m) * conv_kernel(kind, adjoint, p - m, q - n, dx, dy, z, k);
      st(out, i, s);
    }
  });
  return 0;
}

// ------------------------------------------------------------------------------------------
// Chirped z-transform propagation (Methods, "Features and performance": CZT evaluates the
// propagation on an arbitrarily placed and sampled output window; Bluestein method of the
// cited Hu et al.).
//
// Reading: the CZT propagator is the Fresnel form of the RS integral on an explicit output
// window X_p = xo0 + p dxo, Y_q = yo0 + q dyo:
//   U1(X_p, Y_q) = exp(ikz)/(i lambda z) dx dy
//                  sum_{m,n} U0[n][m] exp{ i k [(X_p - x_m)^2 + (Y_q - y_n)^2] / (2z) }.
// The amplitude 1/(i lambda z) is the paraxial limit of the RS kernel amplitude. Bluestein's
// chirp factorisation evaluates this sum exactly; the oracle evaluates it directly.
// Vectorial CZT applies the same -(offset/z) factor as VRS:
//   Ez' = sum [ -(X_p - x_m)/z Ex - (Y_q - y_n)/z Ey ] K.
// Kernel kinds: 0 K, 1 -(X-x)/z K, 2 -(Y-y)/z K, 3 dK/dz, 4 d/dz[-(X-x)/z K],
// 5 d/dz[-(Y-y)/z K], with
//   dK/dz = K [ ik - 1/z - ik ((X-x)^2+(Y-y)^2) / (2 z^2) ].
// ------------------------------------------------------------------------------------------
struct CztGeom {
  int64_t nx, ny, mx, my;
  double dx, dy, x0, y0, dxo, dyo, xo0, yo0, k, lambda, z;
};

static cd czt_pref(const CztGeom& g) {
  cd I(0.0, 1.0);
  return std::exp(I * (g.k * g.z)) / (I * g.lambda * g.z) * (g.dx * g.dy);
}

// Full (non-factored) kernel value, used by the brute-force sum.
static cd czt_kernel_full(const CztGeom& g, int kind, int64_t p, int64_t q, int64_t m, int64_t n) {
  cd I(0.0, 1.0);
  double X = g.xo0 + p * g.dxo, Y = g.yo0 + q * g.dyo;
  double x = g.x0 + m * g.dx, y = g.y0 + n * g.dy;
  double DX = X - x, DY = Y - y, z = g.z;
  cd K = czt_pref(g) * std::exp(I * (g.k * (DX * DX + DY * DY) / (2.0 * z)));
  cd dK = K * (I * g.k - 1.0 / z - I * g.k * (DX * DX + DY * DY) / (2.0 * z * z));
  switch (kind) {
    case 0: return K;
    case 1: return -(DX / z) * K;
    case 2: return -(DY / z) * K;
    case 3: return dK;
    case 4: return -DX * (dK / z - K / (z * z));
    case 5: return -DY * (dK / z - K / (z * z));
  }
  return cd(0.0, 0.0);
}

// Separable realisation: every kernel kind is a short sum of terms c * A(p,m) * B(q,n).
struct SepTerm {
  cd c;
  int ax, by;  // factor selectors: 0 chirp, 1 (X-x) chirp, 2 (X-x)^2 chirp
};

static cd axis_factor(int sel, double D, double k, double z) {
  cd I(0.0, 1.0);
  cd e = std::exp(I * (k * D * D / (2.0 * z)));
  if (sel == 0) return e;
  if (sel == 1) return D * e;
  return D * D * e;
}

static std::vector<SepTerm> czt_terms(const CztGeom& g, int kind) {
  cd I(0.0, 1.0);
  cd P = czt_pref(g);
  double z = g.z, k = g.k;
  std::vector<SepTerm> t;
  cd a = I * k - 1.0 / z;            // dK/dz = K [a - ik (DX^2 + DY^2) / (2 z^2)]
  cd bq = -I * k / (2.0 * z * z);
  switch (kind) {
    case 0: t.push_back({P, 0, 0}); break;
    case 1: t.push_back({-P / z, 1, 0}); break;
    case 2: t.push_back({-P / z, 0, 1}); break;
    case 3:
      t.push_back({P * a, 0, 0});
      t.push_back({P * bq, 2, 0});
      t.push_back({P * bq, 0, 2});
      break;
    case 4:  // -DX (dK/z - K/z^2)
      t.push_back({-P * (a / z - 1.0 / (z * z)), 1, 0});
      t.push_back({-P * bq / z, 3, 0});  // DX^3 factor
      t.push_back({-P * bq / z, 1, 2});
      break;
    case 5:
      t.push_back({-P * (a / z - 1.0 / (z * z)), 0, 1});
      t.push_back({-P * bq / z, 2, 1});
      t.push_back({-P * bq / z, 0, 3});
      break;
  }
  return t;
}

static cd axis_factor_ext(int sel, double D, double k, double z) {
  if (sel == 3) return D * axis_factor(2, D, k, z);
  return axis_factor(sel, D, k, z);
}

// Table F[p][m] = axis factor `sel` of (W0 + p dW) - (s0 + m ds), p < M, m < N.
static std::vector<cd> axis_table(int sel, int64_t M, double W0, double dW, int64_t N, double s0,
                                  double ds, double k, double z) {
  std::vector<cd> F((size_t)(M * N));
  parallel_for(M, [&](int64_t pb, int64_t pe) {
    for (int64_t p = pb; p < pe; ++p)
      for (int64_t m = 0; m < N; ++m)
        F[p * N + m] = axis_factor_ext(sel, (W0 + p * dW) - (s0 + m * ds), k, z);
  });
  return F;
}

static bool czt_geom_ok(const CztGeom& g) {
  return g.nx > 0 && g.ny > 0 && g.mx > 0 && g.my > 0 && g.z > 0.0 && g.lambda > 0.0;
}

static CztGeom make_geom(int64_t nx, int64_t ny, double dx, double dy, double x0, double y0,
                         int64_t mx, int64_t my, double dxo, double dyo, double xo0, double yo0,
                         double wavelength, double z) {
  CztGeom g{nx, ny, mx, my, dx, dy, x0, y0, dxo, dyo, xo0, yo0, 2.0 * PI / wavelength, wavelength, z};
  return g;
}

// Direct separable CZT sum. adjoint == 0: u_in [ny][nx] -> u_out [my][mx].
// adjoint != 0: u_in [my][mx] (window) -> u_out [ny][nx], applying conj of the kernel.
int orc_czt_direct(const double* u_in, double* u_out, int64_t nx, int64_t ny, double dx, double dy,
                   double x0, double y0, int64_t mx, int64_t my, double dxo, double dyo, double xo0,
                   double yo0, double wavelength, double z, int kind, int adjoint) {
  CztGeom g = make_geom(nx, ny, dx, dy, x0, y0, mx, my, dxo, dyo, xo0, yo0, wavelength, z);
  if (!czt_geom_ok(g) || kind < 0 || kind > 5) return -1;
  std::vector<SepTerm> terms = czt_terms(g, kind);
  if (!adjoint) {
    std::vector<cd> out((size_t)(mx * my), cd(0.0, 0.0));
    for (const SepTerm& t : terms) {
      // axis factor tables A[p][m] and B[q][n] of this term
      std::vector<cd> A = axis_table(t.ax, mx, g.xo0, g.dxo, nx, g.x0, g.dx, g.k, g.z);
      std::vector<cd> B = axis_table(t.by, my, g.yo0, g.dyo, ny, g.y0, g.dy, g.k, g.z);
      // pass x: T[n][p] = sum_m U0[n][m] A(p,m)
      std::vector<cd> T((size_t)(ny * mx));
      parallel_for(ny, [&](int64_t nb, int64_t ne) {
        for (int64_t n = nb; n < ne; ++n)
          for (int64_t p = 0; p < mx; ++p) {
            cd s(0.0, 0.0);
            const cd* a = &A[p * nx];
            for (int64_t m = 0; m < nx; ++m) s += ld(u_in, n * nx + m) * a[m];
            T[n * mx + p] = s;
          }
      });
      // pass y: out[q][p] += c * sum_n T[n][p] B(q,n)
      parallel_for(my, [&](int64_t qb, int64_t qe) {
        for (int64_t q = qb; q < qe; ++q) {
          const cd* bq = &B[q * ny];
          for (int64_t p = 0; p < mx; ++p) {
            cd s(0.0, 0.0);
            for (int64_t n = 0; n < ny; ++n) s += T[n * mx + p] * bq[n];
            out[q * mx + p] += t.c * s;
          }
        }
      });
    }
    for (int64_t i = 0; i < mx * my; ++i) st(u_out, i, out[i]);
  } else {
    std::vector<cd> out((size_t)(nx * ny), cd(0.0, 0.0));
    for (const SepTerm& t : terms) {
      std::vector<cd> A = axis_table(t.ax, mx, g.xo0, g.dxo, nx, g.x0, g.dx, g.k, g.z);
      std::vector<cd> B = axis_table(t.by, my, g.yo0, g.dyo, ny, g.y0, g.dy, g.k, g.z);
      // adjoint of pass y: T[n][p] = sum_q conj(B(q,n)) G[q][p]
      std::vector<cd> T((size_t)(ny * mx));
      parallel_for(ny, [&](int64_t nb, int64_t ne) {
        for (int64_t n = nb; n < ne; ++n)
          for (int64_t p = 0; p < mx; ++p) {
            cd s(0.0, 0.0);
            for (int64_t q = 0; q < my; ++q) s += ld(u_in, q * mx + p) * std::conj(B[q * ny + n]);
            T[n * mx + p] = s;
          }
      });
      // adjoint of pass x: out[n][m] += conj(c) sum_p conj(A(p,m)) T[n][p]
      parallel_for(ny, [&](int64_t nb, int64_t ne) {
        for (int64_t n = nb; n < ne; ++n)
          for (int64_t m = 0; m < nx; ++m) {
            cd s(0.0, 0.0);
            for (int64_t p = 0; p < mx; ++p) s += T[n * mx + p] * std::conj(A[p * nx + m]);
            out[n * nx + m] += std::conj(t.c) * s;
          }
      });
    }
    for (int64_t i = 0; i < nx * ny; ++i) st(u_out, i, out[i]);
  }
  return 0;
}

// Brute-force CZT sum with the full, non-factored kernel (tiny sizes only).
int orc_czt_brute(const double* u_in, double* u_out, int64_t nx, int64_t ny, double dx, double dy,
                  double x0, double y0, int64_t mx, int64_t my, double dxo, double dyo, double xo0,
                  double yo0, double wavelength, double z, int kind) {
  CztGeom g = make_geom(nx, ny, dx, dy, x0, y0, mx, my, dxo, dyo, xo0, yo0, wavelength, z);
  if (!czt_geom_ok(g) || kind < 0 || kind > 5) return -1;
  for (int64_t q = 0; q < my; ++q)
    for (int64_t p = 0; p < mx; ++p) {
      cd s(0.0, 0.0);
      for (int64_t n = 0; n < ny; ++n)
        for (int64_t m = 0; m < nx; ++m)
          s += ld(u_in, n * nx + m) * czt_kernel_full(g, kind, p, q, m, n);
      st(u_out, q * mx + p, s);
    }
  return 0;
}

// Direct CZT sum at selected output pixels (p, q), full kernel.
int orc_czt_points(const double* u_in, int64_t nx, int64_t ny, double dx, double dy, double x0,
                   double y0, double dxo, double dyo, double xo0, double yo0, double wavelength,
                   double z, int kind, const int32_t* pts, int64_t npts, double* out) {
  CztGeom g = make_geom(nx, ny, dx, dy, x0, y0, 1, 1, dxo, dyo, xo0, yo0, wavelength, z);
  if (!czt_geom_ok(g) || kind < 0 || kind > 5) return -1;
  parallel_for(npts, [&](int64_t ib, int64_t ie) {
    for (int64_t i = ib; i < ie; ++i) {
      cd s(0.0, 0.0);
      for (int64_t n = 0; n < ny; ++n)
        for (int64_t m = 0; m < nx; ++m)
          s += ld(u_in, n * nx + m) * czt_kernel_full(g, kind, pts[2 * i], pts[2 * i + 1], m, n);
      st(out, i, s);
    }
  });
  return 0;
}

// ------------------------------------------------------------------------------------------
// Optical elements (Methods, "Features and performance": SLMs / super-SLM phase masks,
// polarisers, variable retarders (wave plates), planar lenses).
//
// Readings (the paper names the elements only):
//   SLM          every component times exp(i phi(x,y))
//   super-SLM    Ex times exp(i phi_x), Ey times exp(i phi_y)
//   thin lens    every component times exp(-i k (x^2 + y^2) / (2 f))
//   polariser    J = R(-a) diag(1, 0) R(a)
//   wave plate   J = R(-t) diag(1, exp(i eta)) R(t),   R(t) = [[cos t, sin t], [-sin t, cos t]]
//   to-vector    (Ex, Ey) = (u, 0): an x-polarised scalar field becomes a 2-component field.
// params per element: [f, alpha, eta, theta].
// ------------------------------------------------------------------------------------------
enum { ORC_SLM = 0, ORC_SSLM = 1, ORC_LENS = 2, ORC_POLARIZER = 3, ORC_WAVEPLATE = 4,
       ORC_TO_VECTOR = 5 };

struct Jones {
  cd a, b, c, d;  // [[a, b], [c, d]]
};

static Jones rot(double t) {  // R(t)
  return {cd(std::cos(t), 0), cd(std::sin(t), 0), cd(-std::sin(t), 0), cd(std::cos(t), 0)};
}
static Jones mul(const Jones& x, const Jones& y) {
  return {x.a * y.a + x.b * y.c, x.a * y.b + x.b * y.d, x.c * y.a + x.d * y.c, x.c * y.b + x.d * y.d};
}
static Jones polarizer(double alpha) {
  Jones P{cd(1, 0), cd(0, 0), cd(0, 0), cd(0, 0)};
  return mul(rot(-alpha), mul(P, rot(alpha)));
}
static Jones waveplate(double eta, double theta) {
  Jones D{cd(1, 0), cd(0, 0), cd(0, 0), std::exp(cd(0, eta))};
  return mul(rot(-theta), mul(D, rot(theta)));
}

// Derivatives of the Jones matrices (used by the backward pass).
static Jones dpolarizer_dalpha(double a) {
  // J = [[c^2, cs], [cs, s^2]]
  double c = std::cos(a), s = std::sin(a);
  return {cd(-2 * c * s, 0), cd(c * c - s * s, 0), cd(c * c - s * s, 0), cd(2 * c * s, 0)};
}
static Jones dwaveplate_deta(double eta, double t) {
  // J = R(-t) diag(1, e) R(t); dJ/deta = R(-t) diag(0, i e) R(t)
  Jones D{cd(0, 0), cd(0, 0), cd(0, 0), cd(0, 1) * std::exp(cd(0, eta))};
  return mul(rot(-t), mul(D, rot(t)));
}
static Jones dwaveplate_dtheta(double eta, double t) {
  // d/dt [R(-t) D R(t)] = R'(-t)(-1) D R(t) + R(-t) D R'(t), R'(t) = [[-s, c], [-c, -s]]
  Jones D{cd(1, 0), cd(0, 0), cd(0, 0), std::exp(cd(0, eta))};
  double c = std::cos(t), s = std::sin(t);
  Jones dR_t{cd(-s, 0), cd(c, 0), cd(-c, 0), cd(-s, 0)};           // R'(t)
  Jones dR_mt{cd(-std::sin(-t), 0), cd(std::cos(-t), 0), cd(-std::cos(-t), 0),
              cd(-std::sin(-t), 0)};                               // R'(-t)
  Jones A = mul(dR_mt, mul(D, rot(t)));
  Jones B = mul(rot(-t), mul(D, dR_t));
  return {-A.a + B.a, -A.b + B.b, -A.c + B.c, -A.d + B.d};
}

struct PixelCtx {
  double x, y, k;
};

// Applies element e to the components (c0, c1) at one pixel; ncomp is 1 or 2 on entry and
// is updated by the to-vector element.
static void apply_one(int kind, const double* prm, double phx, double phy, const PixelCtx& px,
                      int& ncomp, cd& c0, cd& c1) {
  switch (kind) {
    case ORC_SLM: {
      cd e = std::exp(cd(0, phx));
      c0 *= e;
      c1 *= e;
      break;
    }
    case ORC_SSLM:
      c0 *= std::exp(cd(0, phx));
      c1 *= std::exp(cd(0, phy));
      break;
    case ORC_LENS: {
      cd e = std::exp(cd(0, -px.k * (px.x * px.x + px.y * px.y) / (2.0 * prm[0])));
      c0 *= e;
      c1 *= e;
      break;
    }
    case ORC_POLARIZER: {
      Jones J = polarizer(prm[1]);
      cd a = J.a * c0 + J.b * c1, b = J.c * c0 + J.d * c1;
      c0 = a;
      c1 = b;
      break;
    }
    case ORC_WAVEPLATE: {
      Jones J = waveplate(prm[2], prm[3]);
      cd a = J.a * c0 + J.b * c1, b = J.c * c0 + J.d * c1;
      c0 = a;
      c1 = b;
      break;
    }
    case ORC_TO_VECTOR:
      ncomp = 2;
      c1 = cd(0, 0);
      break;
  }
}

static bool elements_ok(int comps_in, int n_el, const int32_t* kinds) {
  if (comps_in != 1 && comps_in != 2) return false;
  int c = comps_in;
  for (int i = 0; i < n_el; ++i) {
    int kd = kinds[i];
    if (kd < 0 || kd > 5) return false;
    if ((kd == ORC_SSLM || kd == ORC_POLARIZER || kd == ORC_WAVEPLATE) && c != 2) return false;
    if (kd == ORC_TO_VECTOR) {
      if (c != 1) return false;
      c = 2;
    }
  }
  return true;
}

static int comps_out_of(int comps_in, int n_el, const int32_t* kinds) {
  int c = comps_in;
  for (int i = 0; i < n_el; ++i)
    if (kinds[i] == ORC_TO_VECTOR) c = 2;
  return c;
}

// Forward chain. in: [comps_in][ny][nx]; out: [comps_out][ny][nx].
// phix/phiy: per element pointers to [ny][nx] phase masks (may be null when unused).
int orc_elements_forward(const double* in, double* out, int comps_in, int64_t nx, int64_t ny,
                         double dx, double dy, double x0, double y0, double wavelength, int n_el,
                         const int32_t* kinds, const double* params, const double* const* phix,
                         const double* const* phiy) {
  if (!elements_ok(comps_in, n_el, kinds)) return -1;
  int co = comps_out_of(comps_in, n_el, kinds);
  int64_t P = nx * ny;
  double k = 2.0 * PI / wavelength;
  for (int64_t n = 0; n < ny; ++n)
    for (int64_t m = 0; m < nx; ++m) {
      int64_t i = n * nx + m;
      PixelCtx px{x0 + m * dx, y0 + n * dy, k};
      int nc = comps_in;
      cd c0 = ld(in, i), c1 = comps_in == 2 ? ld(in, P + i) : cd(0, 0);
      for (int e = 0; e < n_el; ++e)
        apply_one(kinds[e], params + 4 * e, phix[e] ? phix[e][i] : 0.0, phiy[e] ? phiy[e][i] : 0.0,
                  px, nc, c0, c1);
      st(out, i, c0);
      if (co == 2) st(out, P + i, c1);
    }
  return 0;
}

// Backward chain: given g_out ([comps_out][ny][nx]) and the forward input, writes
//   g_in [comps_in][ny][nx]      g = J^H g_out per element, in reverse order;
//   g_phix/g_phiy per element    dL/dphi = Im(g_out_e conj(u_out_e)) (summed over components
//                                for an SLM, per component for a super-SLM);
//   g_params [n_el][4]           dL/d{f, alpha, eta, theta} = sum Re(conj(g_out_e) dJ u_in_e).
int orc_elements_backward(const double* g_out, const double* in, double* g_in, int comps_in,
                          int64_t nx, int64_t ny, double dx, double dy, double x0, double y0,
                          double wavelength, int n_el, const int32_t* kinds, const double* params,
                          const double* const* phix, const double* const* phiy,
                          double* const* g_phix, double* const* g_phiy, double* g_params) {
  if (!elements_ok(comps_in, n_el, kinds)) return -1;
  int co = comps_out_of(comps_in, n_el, kinds);
  int64_t P = nx * ny;
  double k = 2.0 * PI / wavelength;
  for (int e = 0; e < 4 * n_el; ++e) g_params[e] = 0.0;
  std::vector<cd> s0(n_el + 1), s1(n_el + 1);
  std::vector<int> nc_at(n_el + 1);
  for (int64_t n = 0; n < ny; ++n)
    for (int64_t m = 0; m < nx; ++m) {
      int64_t i = n * nx + m;
      PixelCtx px{x0 + m * dx, y0 + n * dy, k};
      int nc = comps_in;
      s0[0] = ld(in, i);
      s1[0] = comps_in == 2 ? ld(in, P + i) : cd(0, 0);
      nc_at[0] = nc;
      for (int e = 0; e < n_el; ++e) {
        cd c0 = s0[e], c1 = s1[e];
        apply_one(kinds[e], params + 4 * e, phix[e] ? phix[e][i] : 0.0, phiy[e] ? phiy[e][i] : 0.0,
                  px, nc, c0, c1);
        s0[e + 1] = c0;
        s1[e + 1] = c1;
        nc_at[e + 1] = nc;
      }
      cd g0 = ld(g_out, i), g1 = co == 2 ? ld(g_out, P + i) : cd(0, 0);
      for (int e = n_el - 1; e >= 0; --e) {
        const double* prm = params + 4 * e;
        cd u0 = s0[e], u1 = s1[e], o0 = s0[e + 1], o1 = s1[e + 1];
        switch (kinds[e]) {
          case ORC_SLM: {
            if (g_phix[e]) g_phix[e][i] = std::imag(g0 * std::conj(o0) + g1 * std::conj(o1));
            cd ec = std::exp(cd(0, -(phix[e] ? phix[e][i] : 0.0)));
            g0 *= ec;
            g1 *= ec;
            break;
          }
          case ORC_SSLM: {
            if (g_phix[e]) g_phix[e][i] = std::imag(g0 * std::conj(o0));
            if (g_phiy[e]) g_phiy[e][i] = std::imag(g1 * std::conj(o1));
            g0 *= std::exp(cd(0, -(phix[e] ? phix[e][i] : 0.0)));
            g1 *= std::exp(cd(0, -(phiy[e] ? phiy[e][i] : 0.0)));
            break;
          }
          case ORC_LENS: {
            double r2 = px.x * px.x + px.y * px.y, f = prm[0];
            // d out / d f = out * (i k r2 / (2 f^2))
            cd d = cd(0, k * r2 / (2.0 * f * f));
            g_params[4 * e + 0] += std::real(std::conj(g0) * o0 * d + std::conj(g1) * o1 * d);
            cd ec = std::exp(cd(0, k * r2 / (2.0 * f)));
            g0 *= ec;
            g1 *= ec;
            break;
          }
          case ORC_POLARIZER: {
            Jones J = polarizer(prm[1]), dJ = dpolarizer_dalpha(prm[1]);
            g_params[4 * e + 1] += std::real(std::conj(g0) * (dJ.a * u0 + dJ.b * u1) +
                                             std::conj(g1) * (dJ.c * u0 + dJ.d * u1));
            cd a = std::conj(J.a) * g0 + std::conj(J.c) * g1;
            cd b = std::conj(J.b) * g0 + std::conj(J.d) * g1;
            g0 = a;
            g1 = b;
            break;
          }
          case ORC_WAVEPLATE: {
            Jones J = waveplate(prm[2], prm[3]);
            Jones de = dwaveplate_deta(prm[2], prm[3]), dt = dwaveplate_dtheta(prm[2], prm[3]);
            g_params[4 * e + 2] += std::real(std::conj(g0) * (de.a * u0 + de.b * u1) +
                                             std::conj(g1) * (de.c * u0 + de.d * u1));
            g_params[4 * e + 3] += std::real(std::conj(g0) * (dt.a * u0 + dt.b * u1) +
                                             std::conj(g1) * (dt.c * u0 + dt.d * u1));
            cd a = std::conj(J.a) * g0 + std::conj(J.c) * g1;
            cd b = std::conj(J.b) * g0 + std::conj(J.d) * g1;
            g0 = a;
            g1 = b;
            break;
          }
          case ORC_TO_VECTOR:
            g1 = cd(0, 0);
            break;
        }
      }
      st(g_in, i, g0);
      if (comps_in == 2) st(g_in, P + i, g1);
    }
  return 0;
}

// ------------------------------------------------------------------------------------------
// Camera intensity and losses.
//   Intensity (Results and Methods: radial |Ex|^2+|Ey|^2, longitudinal |Ez|^2, or total):
//       I = sum over the components selected by comp_mask of |E_c|^2.
//   Mode 0, second-moment spot size (reading; the paper's own spot metric is (pi/4) FWHMx FWHMy):
//       P = sum I, xbar = sum I x / P, sigma_x^2 = sum I (x - xbar)^2 / P (same for y),
//       L = sigma_x^2 + sigma_y^2.
//   Mode 1, density loss (Methods, "Loss function"): threshold eps * i_max with a strict ">",
//       I_eps = sum of the pixels above it, Area = their count, L = Area / I_eps.
// ------------------------------------------------------------------------------------------
static void intensity_of(const double* field, int comps, uint32_t mask, int64_t P,
                         std::vector<double>& I) {
  I.assign(P, 0.0);
  for (int c = 0; c < comps; ++c)
    if (mask & (1u << c))
      for (int64_t i = 0; i < P; ++i) I[i] += std::norm(ld(field, (int64_t)c * P + i));
}

int orc_intensity_loss(const double* field, int comps, uint32_t mask, int64_t nx, int64_t ny,
                       double dx, double dy, double x0, double y0, int mode, double eps,
                       double* loss_out, double* intensity_out) {
  if (comps < 1 || comps > 3 || nx < 1 || ny < 1) return -1;
  int64_t P = nx * ny;
  std::vector<double> I;
  intensity_of(field, comps, mask, P, I);
  if (intensity_out)
    for (int64_t i = 0; i < P; ++i) intensity_out[i] = I[i];
  if (mode == 0) {
    double S = 0, Sx = 0, Sy = 0;
    for (int64_t n = 0; n < ny; ++n)
      for (int64_t m = 0; m < nx; ++m) {
        double v = I[n * nx + m];
        S += v;
        Sx += v * (x0 + m * dx);
        Sy += v * (y0 + n * dy);
      }
    double xb = Sx / S, yb = Sy / S, V = 0;
    for (int64_t n = 0; n < ny; ++n)
      for (int64_t m = 0; m < nx; ++m) {
        double ex = x0 + m * dx - xb, ey = y0 + n * dy - yb;
        V += I[n * nx + m] * (ex * ex + ey * ey);
      }
    *loss_out = V / S;
  } else if (mode == 1) {
    double imax = 0;
    for (int64_t i = 0; i < P; ++i) imax = std::max(imax, I[i]);
    double thr = eps * imax, Ie = 0, area = 0;
    for (int64_t i = 0; i < P; ++i)
      if (I[i] > thr) {
        Ie += I[i];
        area += 1.0;
      }
    *loss_out = area / Ie;
  } else {
    return -1;
  }
  return 0;
}

// g_field = dL/dE (torch convention) = 2 g_loss (dL/dI) E on selected components, 0 elsewhere.
//   mode 0: dL/dI = [(x - xbar)^2 + (y - ybar)^2 - L] / P
//   mode 1: dL/dI = -Area / I_eps^2 on pixels above the threshold, 0 elsewhere (the selection,
//           i_max and Area carry no gradient, as with a where-based selection).
int orc_intensity_loss_backward(const double* field, int comps, uint32_t mask, int64_t nx,
                                int64_t ny, double dx, double dy, double x0, double y0, int mode,
                                double eps, double g_loss, double* g_field) {
  if (comps < 1 || comps > 3 || nx < 1 || ny < 1) return -1;
  int64_t P = nx * ny;
  std::vector<double> I, dI(P, 0.0);
  intensity_of(field, comps, mask, P, I);
  if (mode == 0) {
    double S = 0, Sx = 0, Sy = 0;
    for (int64_t n = 0; n < ny; ++n)
      for (int64_t m = 0; m < nx; ++m) {
        double v = I[n * nx + m];
        S += v;
        Sx += v * (x0 + m * dx);
        Sy += v * (y0 + n * dy);
      }
    double xb = Sx / S, yb = Sy / S, V = 0;
    for (int64_t n = 0; n < ny; ++n)
      for (int64_t m = 0; m < nx; ++m) {
        double ex = x0 + m * dx - xb, ey = y0 + n * dy - yb;
        V += I[n * nx + m] * (ex * ex + ey * ey);
      }
    double L = V / S;
    for (int64_t n = 0; n < ny; ++n)
      for (int64_t m = 0; m < nx; ++m) {
        double ex = x0 + m * dx - xb, ey = y0 + n * dy - yb;
        dI[n * nx + m] = (ex * ex + ey * ey - L) / S;
      }
  } else if (mode == 1) {
    double imax = 0;
    for (int64_t i = 0; i < P; ++i) imax = std::max(imax, I[i]);
    double thr = eps * imax, Ie = 0, area = 0;
    for (int64_t i = 0; i < P; ++i)
      if (I[i] > thr) {
        Ie += I[i];
        area += 1.0;
      }
    for (int64_t i = 0; i < P; ++i)
      if (I[i] > thr) dI[i] = -area / (Ie * Ie);
  } else {
    return -1;
  }
  for (int c = 0; c < comps; ++c) {
    bool on = (mask & (1u << c)) != 0;
    for (int64_t i = 0; i < P; ++i) {
      cd E = ld(field, (int64_t)c * P + i);
      st(g_field, (int64_t)c * P + i, on ? 2.0 * g_loss * dI[i] * E : cd(0, 0));
    }
  }
  return 0;
}

// ------------------------------------------------------------------------------------------
// STED effective intensity (Methods, "Stimulated emission depletion model"):
//   I_eff = I_ex [1 - beta (1 - exp(-I_dep / I_ex))], with I_eff = 0 where I_ex = 0 (the
//   limit the paper states).
// ------------------------------------------------------------------------------------------
void orc_sted(const double* i_ex, const double* i_dep, double beta, int64_t n, double* out) {
  for (int64_t i = 0; i < n; ++i)
    out[i] = i_ex[i] > 0.0 ? i_ex[i] * (1.0 - beta * (1.0 - std::exp(-i_dep[i] / i_ex[i]))) : 0.0;
}

// ------------------------------------------------------------------------------------------
// Adam (the paper's optimiser; Kingma & Ba), bias-corrected, step t >= 1:
//   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
//   p -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
// ------------------------------------------------------------------------------------------
void orc_adam(double* p, double* m, double* v, const double* g, int64_t n, double lr, double b1,
              double b2, double eps, int64_t t) {
  double c1 = 1.0 - std::pow(b1, (double)t), c2 = 1.0 - std::pow(b2, (double)t);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    p[i] -= lr * (m[i] / c1) / (std::sqrt(v[i] / c2) + eps);
  }
}

// ------------------------------------------------------------------------------------------
// Losses of an intensity image (the same definitions as above, from I directly), their
// gradients dL/dI, the STED derivative, softmin over detectors, AdamW and MSE.
// ------------------------------------------------------------------------------------------
static double sm_loss_and_grad(const double* I, int64_t nx, int64_t ny, double dx, double dy,
                               double x0, double y0, double* dI) {
  double S = 0, Sx = 0, Sy = 0;
  for (int64_t n = 0; n < ny; ++n)
    for (int64_t m = 0; m < nx; ++m) {
      double v = I[n * nx + m];
      S += v;
      Sx += v * (x0 + m * dx);
      Sy += v * (y0 + n * dy);
    }
  double xb = Sx / S, yb = Sy / S, V = 0;
  for (int64_t n = 0; n < ny; ++n)
    for (int64_t m = 0; m < nx; ++m) {
      double ex = x0 + m * dx - xb, ey = y0 + n * dy - yb;
      V += I[n * nx + m] * (ex * ex + ey * ey);
    }
  double L = V / S;
  if (dI)
    for (int64_t n = 0; n < ny; ++n)
      for (int64_t m = 0; m < nx; ++m) {
        double ex = x0 + m * dx - xb, ey = y0 + n * dy - yb;
        dI[n * nx + m] = (ex * ex + ey * ey - L) / S;
      }
  return L;
}

static double density_loss_and_grad(const double* I, int64_t P, double eps, double* dI) {
  double imax = 0;
  for (int64_t i = 0; i < P; ++i) imax = std::max(imax, I[i]);
  double thr = eps * imax, Ie = 0, area = 0;
  for (int64_t i = 0; i < P; ++i)
    if (I[i] > thr) {
      Ie += I[i];
      area += 1.0;
    }
  if (dI)
    for (int64_t i = 0; i < P; ++i) dI[i] = I[i] > thr ? -area / (Ie * Ie) : 0.0;
  return area / Ie;
}

// Loss of an intensity image (mode 0 second moment, 1 density); dI (nullable) gets dL/dI.
int orc_loss_from_intensity(const double* I, int64_t nx, int64_t ny, double dx, double dy, double x0,
                            double y0, int mode, double eps, double* loss_out, double* dI) {
  if (nx < 1 || ny < 1) return -1;
  if (mode == 0) *loss_out = sm_loss_and_grad(I, nx, ny, dx, dy, x0, y0, dI);
  else if (mode == 1) *loss_out = density_loss_and_grad(I, nx * ny, eps, dI);
  else return -1;
  return 0;
}

// STED derivatives (Methods, "Stimulated emission depletion model", by differentiating the
// effective intensity): with r = I_dep / I_ex,
//   dI_eff/dI_ex  = 1 - beta + beta exp(-r) (1 + r),   dI_eff/dI_dep = -beta exp(-r);
// at I_ex = 0 (where I_eff = 0) the limits for I_dep > 0: (1 - beta, 0).
void orc_sted_backward(const double* i_ex, const double* i_dep, double beta, const double* g_eff,
                       int64_t n, double* g_ex, double* g_dep) {
  for (int64_t i = 0; i < n; ++i) {
    if (i_ex[i] > 0.0) {
      double r = i_dep[i] / i_ex[i], e = std::exp(-r);
      g_ex[i] = g_eff[i] * (1.0 - beta + beta * e * (1.0 + r));
      g_dep[i] = g_eff[i] * (-beta * e);
    } else {
      g_ex[i] = g_eff[i] * (1.0 - beta);
      g_dep[i] = 0.0;
    }
  }
}

// Softmin over detectors (Methods, "Rediscovery through exploration of optical topologies": the
// update follows the detector with the smallest loss through a smooth minimum):
//   softmin(l) = -log(sum_d exp(-beta l_d)) / beta;  weights w_d = d softmin / d l_d
//   = exp(-beta l_d) / sum exp(-beta l) (computed with the minimum subtracted).
void orc_softmin(const double* l, int64_t batch, int64_t n, double beta, double* out, double* w) {
  for (int64_t b = 0; b < batch; ++b) {
    const double* lb = l + b * n;
    double mn = lb[0];
    for (int64_t d = 1; d < n; ++d) mn = std::min(mn, lb[d]);
    double s = 0;
    for (int64_t d = 0; d < n; ++d) s += std::exp(-beta * (lb[d] - mn));
    out[b] = mn - std::log(s) / beta;
    if (w)
      for (int64_t d = 0; d < n; ++d) w[b * n + d] = std::exp(-beta * (lb[d] - mn)) / s;
  }
}

// AdamW (decoupled weight decay, Loshchilov & Hutter): the Adam step of orc_adam plus
// p -= lr * wd * p (using p before the step).
void orc_adamw(double* p, double* m, double* v, const double* g, int64_t n, double lr, double b1,
               double b2, double eps, double wd, int64_t t) {
  double c1 = 1.0 - std::pow(b1, (double)t), c2 = 1.0 - std::pow(b2, (double)t);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    p[i] -= lr * ((m[i] / c1) / (std::sqrt(v[i] / c2) + eps) + wd * p[i]);
  }
}

// Mean squared error between an intensity image and a target (Results, "Data-driven
// rediscovery": L = MSE(I_det, I_GT)); dI (nullable) gets dL/dI = 2 (I - I_GT) / P.
double orc_mse(const double* I, const double* target, int64_t P, double* dI) {
  double s = 0;
  for (int64_t i = 0; i < P; ++i) {
    double d = I[i] - target[i];
    s += d * d;
    if (dI) dI[i] = 2.0 * d / (double)P;
  }
  return s / (double)P;
}

// Angular-spectrum CZT: the exact-RS reading of the chirped z-transform propagator (Methods,
// "Features and performance"; Hu et al.): the angular spectrum of the sampled field, times the
// free-space transfer function, summed back onto an arbitrary output window.
//   U^(f, g) = sum_{n,m} u[n][m] exp(-2 pi i (f x_m + g y_n)),  f = j / (nx dx), g = l / (ny dy),
//              j, l over the signed frequency indices [-n/2, n/2) of an n-point DFT,
//   H = exp(i z kz), kz = sqrt(k^2 - (2 pi f)^2 - (2 pi g)^2) (kz = i sqrt(-...) beyond the
//       light cone: evanescent decay),
//   U1(X_p, Y_q) = 1 / (nx ny) sum_{f,g} U^ H exp(2 pi i (f X_p + g Y_q)).
// kind 0: H; kind 1: dH/dz = i kz H (the distance derivative). adjoint: the conjugate-transpose
// map (window -> input grid). The spectrum uses the FFT (sizes: powers of two); the sums onto the
// window are direct and separable.
static cd as_transfer(double f, double g, double k, double z, int kind) {
  const double a = k * k - 4.0 * PI * PI * (f * f + g * g);
  cd kz = a >= 0.0 ? cd(std::sqrt(a), 0.0) : cd(0.0, std::sqrt(-a));
  cd H = std::exp(cd(0.0, 1.0) * kz * z);
  return kind == 1 ? cd(0.0, 1.0) * kz * H : H;
}

static double as_freq(int64_t k, int64_t n, double d) {  // FFT bin k -> signed frequency
  const int64_t j = k < n / 2 ? k : k - n;
  return (double)j / ((double)n * d);
}

int orc_asczt(const double* u_in, double* u_out, int64_t nx, int64_t ny, double dx, double dy,
              double x0, double y0, int64_t mx, int64_t my, double dxo, double dyo, double xo0,
              double yo0, double wavelength, double z, int kind, int adjoint) {
  if (!is_pow2(nx) || !is_pow2(ny) || mx < 1 || my < 1 || kind < 0 || kind > 1) return -1;
  const double k = 2.0 * PI / wavelength;
  std::vector<double> fx(nx), fy(ny);
  for (int64_t i = 0; i < nx; ++i) fx[i] = as_freq(i, nx, dx);
  for (int64_t i = 0; i < ny; ++i) fy[i] = as_freq(i, ny, dy);
  // window exponentials Ex[p][j] = exp(2 pi i f_j X_p), Ey[q][l] = exp(2 pi i g_l Y_q)
  std::vector<cd> Ex((size_t)(mx * nx)), Ey((size_t)(my * ny));
  for (int64_t p = 0; p < mx; ++p)
    for (int64_t j = 0; j < nx; ++j) Ex[p * nx + j] = std::exp(cd(0.0, 2.0 * PI * fx[j] * (xo0 + p * dxo)));
  for (int64_t q = 0; q < my; ++q)
    for (int64_t l = 0; l < ny; ++l) Ey[q * ny + l] = std::exp(cd(0.0, 2.0 * PI * fy[l] * (yo0 + q * dyo)));
  const double norm = 1.0 / ((double)nx * (double)ny);
  std::vector<cd> W((size_t)(nx * ny));
  if (!adjoint) {
    // spectrum: FFT, then the phase of the grid origin
    for (int64_t i = 0; i < nx * ny; ++i) W[i] = ld(u_in, i);
    fft2_inplace(W, ny, nx, -1);
    for (int64_t l = 0; l < ny; ++l)
      for (int64_t j = 0; j < nx; ++j)
        W[l * nx + j] *= std::exp(cd(0.0, -2.0 * PI * (fx[j] * x0 + fy[l] * y0))) *
                         as_transfer(fx[j], fy[l], k, z, kind);
    // onto the window: V[l][p] = sum_j W[l][j] Ex[p][j]; out[q][p] = norm sum_l V[l][p] Ey[q][l]
    std::vector<cd> V((size_t)(ny * mx));
    parallel_for(ny, [&](int64_t b, int64_t e) {
      for (int64_t l = b; l < e; ++l)
        for (int64_t p = 0; p < mx; ++p) {
          cd s(0.0, 0.0);
          for (int64_t j = 0; j < nx; ++j) s += W[l * nx + j] * Ex[p * nx + j];
          V[l * mx + p] = s;
        }
    });
    parallel_for(my, [&](int64_t b, int64_t e) {
      for (int64_t q = b; q < e; ++q)
        for (int64_t p = 0; p < mx; ++p) {
          cd s(0.0, 0.0);
          for (int64_t l = 0; l < ny; ++l) s += V[l * mx + p] * Ey[q * ny + l];
          st(u_out, q * mx + p, norm * s);
        }
    });
  } else {
    // adjoint of the window sums: V[l][p] = sum_q G[q][p] conj(Ey[q][l]);
    // W[l][j] = norm sum_p V[l][p] conj(Ex[p][j])
    std::vector<cd> V((size_t)(ny * mx));
    parallel_for(ny, [&](int64_t b, int64_t e) {
      for (int64_t l = b; l < e; ++l)
        for (int64_t p = 0; p < mx; ++p) {
          cd s(0.0, 0.0);
          for (int64_t q = 0; q < my; ++q) s += ld(u_in, q * mx + p) * std::conj(Ey[q * ny + l]);
          V[l * mx + p] = s;
        }
    });
    parallel_for(ny, [&](int64_t b, int64_t e) {
      for (int64_t l = b; l < e; ++l)
        for (int64_t j = 0; j < nx; ++j) {
          cd s(0.0, 0.0);
          for (int64_t p = 0; p < mx; ++p) s += V[l * mx + p] * std::conj(Ex[p * nx + j]);
          W[l * nx + j] = norm * s;
        }
    });
    // adjoint of the spectrum step: conj(H) and the conjugate origin phase, then the
    // unnormalised inverse transform
    for (int64_t l = 0; l < ny; ++l)
      for (int64_t j = 0; j < nx; ++j)
        W[l * nx + j] *= std::exp(cd(0.0, 2.0 * PI * (fx[j] * x0 + fy[l] * y0))) *
                         std::conj(as_transfer(fx[j], fy[l], k, z, kind));
    fft2_inplace(W, ny, nx, +1);
    for (int64_t i = 0; i < nx * ny; ++i) st(u_out, i, W[i]);
  }
  return 0;
}

// Lossless, non-polarising beam splitter (Results, "Towards large-scale discovery", and Methods,
// "The large-scale search space": beam splitters with a continuous ratio in [0, 1] connect the
// paths of the optical table). Reading: R is the reflected intensity fraction, amplitudes
// t = sqrt(1 - R), r = sqrt(R), and the reflected amplitude carries the factor i (the symmetric
// unitary convention):  out_t = t a + i r b,  out_r = i r a + t b.  a or b NULL: a zero input.
void orc_beam_splitter(const cd* a, const cd* b, int64_t n, double R, cd* out_t, cd* out_r) {
  const double t = std::sqrt(1.0 - R), r = std::sqrt(R);
  const cd ir(0.0, r);
  for (int64_t i = 0; i < n; ++i) {
    const cd av = a ? a[i] : cd(0.0), bv = b ? b[i] : cd(0.0);
    out_t[i] = t * av + ir * bv;
    out_r[i] = ir * av + t * bv;
  }
}

// Adjoint of orc_beam_splitter (the conjugate transpose of [[t, i r], [i r, t]]):
//   g_a = t g_t - i r g_r,  g_b = -i r g_t + t g_r,
// and dL/dR = Re sum conj(g_t) d out_t/dR + conj(g_r) d out_r/dR with dt/dR = -1/(2t),
// dr/dR = 1/(2r) (unbounded at R = 0 and R = 1). g_t, g_r, a, b may be NULL (zero).
void orc_beam_splitter_backward(const cd* g_t, const cd* g_r, const cd* a, const cd* b, int64_t n,
                                double R, cd* g_a, cd* g_b, double* g_R) {
  const double t = std::sqrt(1.0 - R), r = std::sqrt(R);
  const cd ir(0.0, r);
  const double dt = -0.5 / t, dr = 0.5 / r;
  double acc = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    const cd gt = g_t ? g_t[i] : cd(0.0), gr = g_r ? g_r[i] : cd(0.0);
    const cd av = a ? a[i] : cd(0.0), bv = b ? b[i] : cd(0.0);
    if (g_a) g_a[i] = t * gt - ir * gr;
    if (g_b) g_b[i] = -ir * gt + t * gr;
    if (g_R) {
      const cd dot = dt * av + cd(0.0, dr) * bv, dor = cd(0.0, dr) * av + dt * bv;
      acc += std::real(std::conj(gt) * dot) + std::real(std::conj(gr) * dor);
    }
  }
  if (g_R) *g_R = acc;
}

}  // extern "C"
