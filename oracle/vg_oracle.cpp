// CPU oracle for the tile-based differentiable Gaussian rasteriser R(G, C) and its loss.
//
// TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's CPU
// baseline may load this library; the product path never calls it.  It shares no code,
// header or constant with the CUDA library.
//
// What it computes (paper Sec. 3): every 3D Gaussian (position, anisotropic covariance from
// scale + rotation, opacity, spherical-harmonic colour) is projected to a 2D Gaussian (EWA
// splatting), assigned to the image tiles it overlaps, sorted by depth within each tile, and
// alpha-blended front to back into the rendered image I^r = R(G, C_i); the adjoint gives the
// gradient of a loss on I^r with respect to every raw parameter (the "differentiable
// rasterizer" of Sec. 3).  The loss is Eq. 1: (1 - lambda) L1 + lambda D-SSIM.
// The rasteriser constants (0.3 low-pass dilation, alpha clamp 0.99, skip alpha < 1/255,
// stop when transmittance < 1e-4, 16x16 tiles, SH degree 0..3) are the method's settings
// and arrive through OrOpts.
//
// Precision: FP64 throughout, except the quantities that decide integers.  The sort key
// (tile, depth) and the tile rectangle are integer results decided by floating point, so
// they are decided in FP32 exactly as the GPU decides them:
//   depth   = fma(R20, x, fma(R21, y, fma(R22, z, t2)))  in float
//   u       = fma(fx, px / pz, cx), v likewise            in float (IEEE division)
//   x_lo    = max(0, ceil(u - r)), x_hi = min(W-1, floor(u + r)) with r rounded to float
// Decisions whose FP64 margin is inside a small band are reported as ambiguous so that tests
// can exclude exactly those.
//
// Readings where the paper is silent (each also stated in the design notes):
//   pixel (i, j) is sampled at image-plane (i, j); camera frame +z forward, +y down;
//   the Gaussian that would take T below t_min is not blended (stop_rule 0; 1 = blend then
//   stop); a Gaussian touches a tile iff the closed box [u-r, u+r] x [v-r, v+r], r = 3
//   sqrt(lambda_max), contains a pixel sample of that tile inside the image; J is evaluated
//   at view-space x/z, y/z clamped to +-guard * (W/2)/fx (resp. H/2 / fy); colours are
//   clamped at 0 after the +0.5 offset; the alpha clamp has zero derivative where active;
//   D-SSIM = 1 - SSIM with an 11x11 Gaussian window (sigma 1.5), zero padding, C1 = 0.01^2,
//   C2 = 0.03^2, L1 is the mean over 3 H W.
#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {

struct OrCamera {
  int32_t width, height;
  double fx, fy, cx, cy;
  double Rt[12];        // row-major 3x4 [R | t], world -> camera
  double cam_pos[3];    // camera centre in world coordinates (SH view direction)
  double near_plane;
};

struct OrOpts {
  int32_t tile;          // tile edge in pixels
  int32_t stop_rule;     // 0: not blended when T would drop below t_min; 1: blended, then stop
  double bg[3];
  double dilation, alpha_max, alpha_min, t_min, guard;
  double band_alpha;     // relative band around alpha_min / alpha_max
  double band_t;         // relative band around t_min
  double band_power;     // relative band of power around 0
  double band_rect;      // relative band (times r) of the rectangle decisions
  int32_t n_threads;
  int32_t pad_;
  const uint8_t* tile_mask;   // optional, [tiles]: render only tiles with a non-zero entry
};

struct OrScene {
  int64_t n;
  int32_t sh_degree;
  int32_t pad_;
  const double* means;        // [n,3]
  const double* log_scales;   // [n,3]
  const double* quats;        // [n,4] (w,x,y,z)
  const double* logits;       // [n]
  const double* sh;           // [n,K,3]
};

}  // extern "C"

namespace {

constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------------------------
// Real spherical harmonics, degree <= 3, from their definition
//   Y_l^0  = K_l^0 P_l(cos th)
//   Y_l^m  = sqrt2 K_l^m cos(m ph) P_l^m(cos th)      (m > 0)
//   Y_l^-m = sqrt2 K_l^m sin(m ph) P_l^m(cos th)      (m > 0)
// with K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) and P_l^m(z) = (-1)^m (1-z^2)^(m/2) d^m P_l/dz^m
// (Condon-Shortley phase).  On the unit sphere sin^m(th) e^{i m ph} = (x + i y)^m, so each
// basis function is the polynomial sqrt2 K (-1)^m {Re,Im}((x+iy)^m) P_l^(m)(z); index l^2+l+m.
// ---------------------------------------------------------------------------------------------
struct Poly { double c[4] = {0, 0, 0, 0}; };   // coefficients of 1, z, z^2, z^3

Poly legendre(int l) {
  Poly p0, p1;
  p0.c[0] = 1.0;
  p1.c[1] = 1.0;
  if (l == 0) return p0;
  for (int n = 1; n < l; ++n) {   // (n+1) P_{n+1} = (2n+1) z P_n - n P_{n-1}
    Poly p2;
    for (int k = 0; k < 3; ++k) p2.c[k + 1] += (2.0 * n + 1.0) * p1.c[k];
    for (int k = 0; k < 4; ++k) p2.c[k] -= n * p0.c[k];
    for (int k = 0; k < 4; ++k) p2.c[k] /= (n + 1.0);
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

Poly deriv(const Poly& p) {
  Poly d;
  for (int k = 1; k < 4; ++k) d.c[k - 1] = k * p.c[k];
  return d;
}

double peval(const Poly& p, double z) { return p.c[0] + z * (p.c[1] + z * (p.c[2] + z * p.c[3])); }

double factorial(int n) { double f = 1; for (int i = 2; i <= n; ++i) f *= i; return f; }

std::complex<double> ipow(std::complex<double> w, int m) {
  std::complex<double> r(1.0, 0.0);
  for (int k = 0; k < m; ++k) r *= w;
  return r;
}

// Y[k] and the Euclidean gradient dY[k][3] of the polynomial form at direction d.
void sh_basis(int degree, const double d[3], double* Y, double (*dY)[3]) {
  const std::complex<double> w(d[0], d[1]);
  for (int l = 0; l <= degree; ++l) {
    Poly P = legendre(l);
    for (int m = 0; m <= l; ++m) {
      Poly Q = P;
      for (int k = 0; k < m; ++k) Q = deriv(Q);
      Poly dQ = deriv(Q);
      double K = std::sqrt((2.0 * l + 1.0) / (4.0 * kPi) * factorial(l - m) / factorial(l + m));
      double sign = (m % 2) ? -1.0 : 1.0;
      double q = peval(Q, d[2]), dq = peval(dQ, d[2]);
      std::complex<double> wm = ipow(w, m);
      std::complex<double> wm1 = m > 0 ? ipow(w, m - 1) : std::complex<double>(0, 0);
      if (m == 0) {
        int k = l * l + l;
        Y[k] = K * q;
        if (dY) { dY[k][0] = 0; dY[k][1] = 0; dY[k][2] = K * dq; }
        continue;
      }
      double a = std::sqrt(2.0) * K * sign;
      // Re((x+iy)^m): d/dx = m Re(w^{m-1}), d/dy = -m Im(w^{m-1})
      // Im((x+iy)^m): d/dx = m Im(w^{m-1}), d/dy =  m Re(w^{m-1})
      int kp = l * l + l + m, kn = l * l + l - m;
      Y[kp] = a * wm.real() * q;
      Y[kn] = a * wm.imag() * q;
      if (dY) {
        dY[kp][0] = a * m * wm1.real() * q;
        dY[kp][1] = -a * m * wm1.imag() * q;
        dY[kp][2] = a * wm.real() * dq;
        dY[kn][0] = a * m * wm1.imag() * q;
        dY[kn][1] = a * m * wm1.real() * q;
        dY[kn][2] = a * wm.imag() * dq;
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// small dense helpers (row-major)
// ---------------------------------------------------------------------------------------------
void matmul(const double* A, const double* B, double* C, int n, int k, int m) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j) {
      double s = 0;
      for (int t = 0; t < k; ++t) s += A[i * k + t] * B[t * m + j];
      C[i * m + j] = s;
    }
}
void transpose(const double* A, double* At, int n, int m) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j) At[j * n + i] = A[i * m + j];
}

// Rotation matrix of a unit quaternion (w, x, y, z) and its partial derivatives.
void quat_to_rot(const double q[4], double R[9]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}
void quat_to_rot_partials(const double q[4], double dR[4][9]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  double Dw[9] = {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0};
  double Dx[9] = {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x};
  double Dy[9] = {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y};
  double Dz[9] = {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0};
  std::memcpy(dR[0], Dw, sizeof Dw); std::memcpy(dR[1], Dx, sizeof Dx);
  std::memcpy(dR[2], Dy, sizeof Dy); std::memcpy(dR[3], Dz, sizeof Dz);
}

uint32_t float_bits(float f) { uint32_t u; std::memcpy(&u, &f, 4); return u; }

// One FP32 unit in the last place of |x|.
double ulp32(double x) {
  float f = (float)std::fabs(x);
  if (f < 1e-30f) f = 1e-30f;
  return (double)(std::nextafter(f, INFINITY) - f);
}

// ---------------------------------------------------------------------------------------------
// per-Gaussian projection record
// ---------------------------------------------------------------------------------------------
struct Rec {
  bool valid = false;       // passed the near-plane, quaternion and determinant culls
  bool visible = false;     // valid and the tile rectangle is not empty
  double m[3], p[3], s[3], qn[4], qnorm, Rq[9], Sigma[9], W[9], J[6];
  bool clx = false, cly = false;  // guard-band clamp active on x / y
  double u, v, A, B, C, det, a, b, c, r, o;
  float depth32 = 0, u32 = 0, v32 = 0, r32 = 0;
  int tx0 = 0, tx1 = -1, ty0 = 0, ty1 = -1;          // inclusive tile rectangle
  int atx0 = 0, atx1 = -1, aty0 = 0, aty1 = -1;      // union of both possible rectangles
  int stx0 = 0, stx1 = -1, sty0 = 0, sty1 = -1;      // intersection of both possible rectangles
  bool rect_amb = false;
  double dirv[3], dirlen, d[3], pre[3], rgb[3];
  bool grad_amb = false;    // a gradient-only decision (clamps) sits inside its band
};

struct Pixel { double T; int32_t last; };

struct State {
  OrScene sc;
  OrCamera cam;
  OrOpts op;
  int K, tiles_x, tiles_y;
  std::vector<Rec> rec;
  std::vector<uint64_t> keys;
  std::vector<uint32_t> vals;
  std::vector<int32_t> ranges;   // [tiles, 2]
  std::vector<double> image;     // [3,H,W]
  std::vector<double> Tfin;      // [H,W]
  std::vector<int32_t> last;     // [H,W]
  std::vector<uint8_t> amb_pix;  // [H,W]
  std::vector<uint8_t> rendered_tile;
  int64_t n_eval = 0, n_blend = 0;
  uint64_t decision_hash = 0;
};

// Decide one rectangle edge in FP32: lower = max(0, ceil(u - r)), upper = min(L-1, floor(u + r)).
int rect_lo(float u, float r, int L) {
  float f = u - r;
  if (!(f > -1.0f)) return 0;
  if (f >= (float)L) return L;
  return std::max(0, (int)std::ceil(f));
}
int rect_hi(float u, float r, int L) {
  float f = u + r;
  if (!(f >= 0.0f)) return -1;
  if (f >= (float)L) return L - 1;
  return std::min(L - 1, (int)std::floor(f));
}

void project(State& S, int64_t i) {
  Rec& g = S.rec[i];
  const OrScene& sc = S.sc;
  const OrCamera& cm = S.cam;
  const OrOpts& op = S.op;
  for (int k = 0; k < 3; ++k) g.m[k] = sc.means[3 * i + k];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) g.W[3 * r + c] = cm.Rt[4 * r + c];
  // view space, FP64
  for (int r = 0; r < 3; ++r)
    g.p[r] = cm.Rt[4 * r + 0] * g.m[0] + cm.Rt[4 * r + 1] * g.m[1] + cm.Rt[4 * r + 2] * g.m[2] + cm.Rt[4 * r + 3];
  // key-defining quantities in FP32 with the stated operation order
  float mf[3] = {(float)g.m[0], (float)g.m[1], (float)g.m[2]};
  float Rf[12];
  for (int k = 0; k < 12; ++k) Rf[k] = (float)cm.Rt[k];
  float pf[3];
  for (int r = 0; r < 3; ++r)
    pf[r] = std::fma(Rf[4 * r + 0], mf[0], std::fma(Rf[4 * r + 1], mf[1], std::fma(Rf[4 * r + 2], mf[2], Rf[4 * r + 3])));
  if (!(pf[2] > (float)cm.near_plane)) return;
  g.depth32 = pf[2];
  g.u32 = std::fma((float)cm.fx, pf[0] / pf[2], (float)cm.cx);
  g.v32 = std::fma((float)cm.fy, pf[1] / pf[2], (float)cm.cy);
  // rotation and scale
  double qq = 0;
  for (int k = 0; k < 4; ++k) qq += sc.quats[4 * i + k] * sc.quats[4 * i + k];
  g.qnorm = std::sqrt(qq);
  if (!(g.qnorm > 0)) return;
  for (int k = 0; k < 4; ++k) g.qn[k] = sc.quats[4 * i + k] / g.qnorm;
  quat_to_rot(g.qn, g.Rq);
  for (int k = 0; k < 3; ++k) g.s[k] = std::exp(sc.log_scales[3 * i + k]);
  double M[9], Mt[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) M[3 * r + c] = g.Rq[3 * r + c] * g.s[c];
  transpose(M, Mt, 3, 3);
  matmul(M, Mt, g.Sigma, 3, 3, 3);
  // Jacobian of the perspective projection at the guard-band clamped point
  double z = g.p[2];
  double limx = op.guard * 0.5 * cm.width / cm.fx, limy = op.guard * 0.5 * cm.height / cm.fy;
  double xz = g.p[0] / z, yz = g.p[1] / z;
  double xzc = std::min(limx, std::max(-limx, xz)), yzc = std::min(limy, std::max(-limy, yz));
  g.clx = (xz != xzc);
  g.cly = (yz != yzc);
  if (std::fabs(std::fabs(xz) - limx) < 1e-9 * limx || std::fabs(std::fabs(yz) - limy) < 1e-9 * limy) g.grad_amb = true;
  double J[6] = {cm.fx / z, 0, -cm.fx * xzc / z, 0, cm.fy / z, -cm.fy * yzc / z};
  std::memcpy(g.J, J, sizeof J);
  double T[6], Tt[6], TS[6], S2[4];
  matmul(J, g.W, T, 2, 3, 3);
  transpose(T, Tt, 2, 3);
  matmul(T, g.Sigma, TS, 2, 3, 3);
  matmul(TS, Tt, S2, 2, 3, 2);
  g.A = S2[0] + op.dilation;
  g.B = S2[1];
  g.C = S2[3] + op.dilation;
  g.det = g.A * g.C - g.B * g.B;
  if (!(g.det > 0)) return;
  g.a = g.C / g.det;
  g.b = -g.B / g.det;
  g.c = g.A / g.det;
  double mid = 0.5 * (g.A + g.C);
  double lmax = mid + std::sqrt(std::max(0.0, mid * mid - g.det));
  g.r = 3.0 * std::sqrt(lmax);
  g.u = cm.fx * g.p[0] / z + cm.cx;
  g.v = cm.fy * g.p[1] / z + cm.cy;
  g.o = 1.0 / (1.0 + std::exp(-sc.logits[i]));
  // colour from spherical harmonics at the viewing direction
  double dd = 0;
  for (int k = 0; k < 3; ++k) { g.dirv[k] = g.m[k] - cm.cam_pos[k]; dd += g.dirv[k] * g.dirv[k]; }
  g.dirlen = std::sqrt(dd);
  for (int k = 0; k < 3; ++k) g.d[k] = g.dirv[k] / g.dirlen;
  double Y[16];
  sh_basis(sc.sh_degree, g.d, Y, nullptr);
  for (int ch = 0; ch < 3; ++ch) {
    double acc = 0;
    for (int k = 0; k < S.K; ++k) acc += sc.sh[(i * S.K + k) * 3 + ch] * Y[k];
    g.pre[ch] = acc + 0.5;
    g.rgb[ch] = std::max(0.0, g.pre[ch]);
    if (std::fabs(g.pre[ch]) < 1e-7) g.grad_amb = true;
  }
  g.valid = true;
  // tile rectangle, decided in FP32
  g.r32 = (float)g.r;
  int W = cm.width, H = cm.height, TS_ = op.tile;
  int xlo = rect_lo(g.u32, g.r32, W), xhi = rect_hi(g.u32, g.r32, W);
  int ylo = rect_lo(g.v32, g.r32, H), yhi = rect_hi(g.v32, g.r32, H);
  if (xlo <= xhi && ylo <= yhi) {
    g.visible = true;
    g.tx0 = xlo / TS_; g.tx1 = xhi / TS_; g.ty0 = ylo / TS_; g.ty1 = yhi / TS_;
  }
  // ambiguity of the four edge decisions: both sides agree on u32/v32 exactly, but r is computed
  // through exp/sqrt chains whose last bits may differ.  Shift r by the band both ways.
  double band = op.band_rect * g.r + 4.0 * ulp32(std::fabs(g.u32) + g.r);
  float rlo = (float)std::max(0.0, g.r - band), rhi = (float)(g.r + band);
  int ax0 = rect_lo(g.u32, rhi, W), ax1 = rect_hi(g.u32, rhi, W), ay0 = rect_lo(g.v32, rhi, H), ay1 = rect_hi(g.v32, rhi, H);
  int bx0 = rect_lo(g.u32, rlo, W), bx1 = rect_hi(g.u32, rlo, W), by0 = rect_lo(g.v32, rlo, H), by1 = rect_hi(g.v32, rlo, H);
  bool big_ne = ax0 <= ax1 && ay0 <= ay1, small_ne = bx0 <= bx1 && by0 <= by1;
  if (big_ne) {
    g.atx0 = ax0 / TS_; g.atx1 = ax1 / TS_; g.aty0 = ay0 / TS_; g.aty1 = ay1 / TS_;
    bool same_small = small_ne && bx0 / TS_ == g.atx0 && bx1 / TS_ == g.atx1 && by0 / TS_ == g.aty0 && by1 / TS_ == g.aty1;
    g.rect_amb = !same_small;
    if (small_ne) { g.stx0 = bx0 / TS_; g.stx1 = bx1 / TS_; g.sty0 = by0 / TS_; g.sty1 = by1 / TS_; }
  }
}

inline uint64_t mix(uint64_t h, uint64_t v) { h ^= v + 0x9e3779b97f4a7c15ULL + (h << 6) + (h >> 2); return h; }

// Forward compositing of one tile.  When `trace` is given it receives (list position, alpha,
// T before, G, clamped) for every blended Gaussian of pixel (tx_pix, ty_pix).
struct Step { int32_t pos; uint32_t g; double alpha, Tb, G; bool clamped; };

// `over`, when given, replaces the record of Gaussian `over_id` (finite differences re-project
// one Gaussian and composite its tiles again with everything else unchanged).
void render_pixel(const State& S, int x, int y, int tile, double* C, double* Tout, int32_t* lastout,
                  bool* amb, int64_t* n_eval, int64_t* n_blend, uint64_t* h, std::vector<Step>* trace,
                  const Rec* over = nullptr, uint32_t over_id = 0xFFFFFFFFu) {
  const OrOpts& op = S.op;
  int32_t s0 = S.ranges[2 * tile], s1 = S.ranges[2 * tile + 1];
  double T = 1.0;
  C[0] = C[1] = C[2] = 0.0;
  int32_t last = 0;
  for (int32_t j = s0; j < s1; ++j) {
    const Rec& g = (over && S.vals[j] == over_id) ? *over : S.rec[S.vals[j]];
    ++*n_eval;
    double dx = x - g.u, dy = y - g.v;
    double qa = 0.5 * g.a * dx * dx, qc = 0.5 * g.c * dy * dy, qb = g.b * dx * dy;
    double power = -qa - qc - qb;
    double terms = qa + qc + std::fabs(qb);
    if (terms > 0 && std::fabs(power) <= op.band_power * terms) *amb = true;
    if (power > 0) { *h = mix(*h, 1); continue; }
    double G = std::exp(power);
    double araw = g.o * G;
    double alpha = std::min(op.alpha_max, araw);
    if (std::fabs(araw - op.alpha_min) <= op.band_alpha * op.alpha_min) *amb = true;
    if (alpha < op.alpha_min) { *h = mix(*h, 2); continue; }
    double Tn = T * (1.0 - alpha);
    if (std::fabs(Tn - op.t_min) <= op.band_t * op.t_min) *amb = true;
    bool stop = Tn < op.t_min;
    if (stop && op.stop_rule == 0) { *h = mix(*h, 3); break; }
    bool clamped = araw >= op.alpha_max;
    if (trace) trace->push_back(Step{j - s0, S.vals[j], alpha, T, G, clamped});
    for (int ch = 0; ch < 3; ++ch) C[ch] += g.rgb[ch] * alpha * T;
    T = Tn;
    last = j - s0 + 1;
    ++*n_blend;
    *h = mix(*h, 4 + 2 * (uint64_t)clamped);
    if (stop) break;
  }
  *Tout = T;
  *lastout = last;
}

// Stable sort of the (key, Gaussian id) pairs by key, in emission order for equal keys, and the
// range [first, last + 1) of every tile's run in the sorted keys ((0, 0) for a tile with none).
void sort_keyed_pairs(std::vector<uint64_t>& keys, std::vector<uint32_t>& vals, int tiles,
                      std::vector<int32_t>& ranges) {
  std::vector<size_t> order(keys.size());
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return keys[a] < keys[b]; });
  std::vector<uint64_t> k2(order.size());
  std::vector<uint32_t> v2(order.size());
  for (size_t j = 0; j < order.size(); ++j) { k2[j] = keys[order[j]]; v2[j] = vals[order[j]]; }
  keys.swap(k2);
  vals.swap(v2);
  ranges.assign(2 * (size_t)tiles, 0);
  for (size_t j = 0; j < keys.size(); ++j) {
    int t = (int)(keys[j] >> 32);
    if (j == 0 || (int)(keys[j - 1] >> 32) != t) ranges[2 * t] = (int32_t)j;
    ranges[2 * t + 1] = (int32_t)j + 1;
  }
}

// One key per (Gaussian, tile of its rectangle): (tile id << 32) | FP32 depth bits, emitted in
// Gaussian index order with the rectangle's tiles row-major.
void emit_keys(std::vector<uint64_t>& keys, std::vector<uint32_t>& vals, uint32_t id, int tx0, int tx1, int ty0,
               int ty1, int tiles_x, float depth32) {
  for (int ty = ty0; ty <= ty1; ++ty)
    for (int tx = tx0; tx <= tx1; ++tx) {
      uint64_t tile = (uint64_t)ty * tiles_x + tx;
      keys.push_back((tile << 32) | float_bits(depth32));
      vals.push_back(id);
    }
}

void build_pairs(State& S) {
  int64_t n = S.sc.n;
  S.keys.clear();
  S.vals.clear();
  for (int64_t i = 0; i < n; ++i) {
    const Rec& g = S.rec[i];
    if (!g.visible) continue;
    emit_keys(S.keys, S.vals, (uint32_t)i, g.tx0, g.tx1, g.ty0, g.ty1, S.tiles_x, g.depth32);
  }
  sort_keyed_pairs(S.keys, S.vals, S.tiles_x * S.tiles_y, S.ranges);
}

void set_threads(const OrOpts& op) {
#ifdef _OPENMP
  if (op.n_threads > 0) omp_set_num_threads(op.n_threads);
#else
  (void)op;
#endif
}

}  // namespace

extern "C" {

// Tile lists from given FP32 decision inputs: uvrd[i] = (u, v, r, depth) of Gaussian i, r < 0 for
// a Gaussian culled before its rectangle.  The rectangle edges (closed box [u - r, u + r] x
// [v - r, v + r] against the pixel samples inside a W x H image), the keys and the stable sort
// are the forward pass's own (rect_lo / rect_hi, emit_keys, sort_keyed_pairs), so feeding another
// implementation's FP32 (u, v, r, depth) checks its key generation, sort and ranges alone.
// Returns the number of pairs P; keys [P], vals [P] and ranges [tiles, 2] are written only when
// P <= cap.
int64_t or_pairs_from_fp32(int64_t n, const float* uvrd, int W, int H, int tile, int64_t cap, uint64_t* keys_out,
                           uint32_t* vals_out, int32_t* ranges_out) {
  const int tiles_x = (W + tile - 1) / tile, tiles_y = (H + tile - 1) / tile;
  std::vector<uint64_t> keys;
  std::vector<uint32_t> vals;
  for (int64_t i = 0; i < n; ++i) {
    const float u = uvrd[4 * i], v = uvrd[4 * i + 1], r = uvrd[4 * i + 2], depth = uvrd[4 * i + 3];
    if (!(r >= 0.0f)) continue;
    int xlo = rect_lo(u, r, W), xhi = rect_hi(u, r, W), ylo = rect_lo(v, r, H), yhi = rect_hi(v, r, H);
    if (xlo > xhi || ylo > yhi) continue;
    emit_keys(keys, vals, (uint32_t)i, xlo / tile, xhi / tile, ylo / tile, yhi / tile, tiles_x, depth);
  }
  const int64_t P = (int64_t)keys.size();
  if (P > cap) return P;
  std::vector<int32_t> ranges;
  sort_keyed_pairs(keys, vals, tiles_x * tiles_y, ranges);
  std::memcpy(keys_out, keys.data(), keys.size() * sizeof(uint64_t));
  std::memcpy(vals_out, vals.data(), vals.size() * sizeof(uint32_t));
  std::memcpy(ranges_out, ranges.data(), ranges.size() * sizeof(int32_t));
  return P;
}

int or_sh_basis(int degree, const double* d, double* Y, double* dY) {
  double dy[16][3];
  sh_basis(degree, d, Y, dY ? dy : nullptr);
  if (dY) for (int k = 0; k < (degree + 1) * (degree + 1); ++k) for (int c = 0; c < 3; ++c) dY[3 * k + c] = dy[k][c];
  return 0;
}

// Runs the whole forward pass; returns an opaque handle (free with or_free).
void* or_forward(const OrScene* sc, const OrCamera* cam, const OrOpts* op) {
  State* S = new State();
  S->sc = *sc;
  S->cam = *cam;
  S->op = *op;
  S->op.tile_mask = nullptr;
  S->K = (sc->sh_degree + 1) * (sc->sh_degree + 1);
  int W = cam->width, H = cam->height, TS = op->tile;
  S->tiles_x = (W + TS - 1) / TS;
  S->tiles_y = (H + TS - 1) / TS;
  int tiles = S->tiles_x * S->tiles_y;
  set_threads(*op);
  S->rec.assign(sc->n, Rec());
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t i = 0; i < sc->n; ++i) project(*S, i);
  build_pairs(*S);
  S->image.assign(3 * (size_t)W * H, 0.0);
  S->Tfin.assign((size_t)W * H, 1.0);
  S->last.assign((size_t)W * H, 0);
  S->amb_pix.assign((size_t)W * H, 0);
  S->rendered_tile.assign(tiles, 1);
  if (op->tile_mask)
    for (int t = 0; t < tiles; ++t) S->rendered_tile[t] = op->tile_mask[t] ? 1 : 0;
  std::vector<uint64_t> tile_hash(tiles, 0);
  int64_t ev = 0, bl = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : ev, bl)
  for (int t = 0; t < tiles; ++t) {
    if (!S->rendered_tile[t]) continue;
    int tx = t % S->tiles_x, ty = t / S->tiles_x;
    uint64_t h = 0;
    for (int y = ty * TS; y < std::min(H, (ty + 1) * TS); ++y)
      for (int x = tx * TS; x < std::min(W, (tx + 1) * TS); ++x) {
        double C[3], T;
        int32_t last;
        bool amb = false;
        render_pixel(*S, x, y, t, C, &T, &last, &amb, &ev, &bl, &h, nullptr);
        size_t p = (size_t)y * W + x;
        for (int ch = 0; ch < 3; ++ch) S->image[(size_t)ch * W * H + p] = C[ch] + T * op->bg[ch];
        S->Tfin[p] = T;
        S->last[p] = last;
        S->amb_pix[p] = amb ? 1 : 0;
      }
    tile_hash[t] = h;
  }
  S->n_eval = ev;
  S->n_blend = bl;
  // pixels that a rectangle-edge flip could change: tiles in the union rectangle but not in the
  // decided one (or the reverse) where the Gaussian could reach alpha_min
  for (int64_t i = 0; i < sc->n; ++i) {
    const Rec& g = S->rec[i];
    if (!g.valid || !g.rect_amb) continue;
    for (int ty = g.aty0; ty <= g.aty1; ++ty)
      for (int tx = g.atx0; tx <= g.atx1; ++tx) {
        bool core = tx >= g.stx0 && tx <= g.stx1 && ty >= g.sty0 && ty <= g.sty1;
        if (core) continue;   // in both possible rectangles: unaffected by the flip
        for (int y = ty * TS; y < std::min(H, (ty + 1) * TS); ++y)
          for (int x = tx * TS; x < std::min(W, (tx + 1) * TS); ++x) {
            double dx = x - g.u, dy = y - g.v;
            double power = -0.5 * (g.a * dx * dx + g.c * dy * dy) - g.b * dx * dy;
            if (g.o * std::exp(power) >= op->alpha_min * (1.0 - op->band_alpha)) S->amb_pix[(size_t)y * W + x] = 1;
          }
      }
  }
  uint64_t h = 0;
  for (int t = 0; t < tiles; ++t) h = mix(h, tile_hash[t]);
  for (size_t j = 0; j < S->keys.size(); ++j) h = mix(h, S->keys[j] >> 32);
  for (int64_t i = 0; i < sc->n; ++i) {
    const Rec& g = S->rec[i];
    h = mix(h, (uint64_t)g.valid + 2 * (uint64_t)g.clx + 4 * (uint64_t)g.cly);
    for (int ch = 0; ch < 3; ++ch) h = mix(h, g.pre[ch] > 0);
  }
  S->decision_hash = h;
  return S;
}

void or_free(void* h) { delete (State*)h; }

int64_t or_num_pairs(void* h) { return (int64_t)((State*)h)->keys.size(); }

void or_stats(void* h, int64_t* out /*[4]: evaluations, blends, visible, ambiguous pixels*/) {
  State* S = (State*)h;
  int64_t vis = 0, amb = 0;
  for (auto& g : S->rec) vis += g.visible;
  for (auto a : S->amb_pix) amb += a;
  out[0] = S->n_eval; out[1] = S->n_blend; out[2] = vis; out[3] = amb;
}

uint64_t or_decision_hash(void* h) { return ((State*)h)->decision_hash; }

void or_get_image(void* h, double* img, double* T, int32_t* last, uint8_t* amb) {
  State* S = (State*)h;
  std::memcpy(img, S->image.data(), S->image.size() * sizeof(double));
  if (T) std::memcpy(T, S->Tfin.data(), S->Tfin.size() * sizeof(double));
  if (last) std::memcpy(last, S->last.data(), S->last.size() * sizeof(int32_t));
  if (amb) std::memcpy(amb, S->amb_pix.data(), S->amb_pix.size());
}

void or_get_pairs(void* h, uint64_t* keys, uint32_t* vals, int32_t* ranges) {
  State* S = (State*)h;
  if (keys) std::memcpy(keys, S->keys.data(), S->keys.size() * sizeof(uint64_t));
  if (vals) std::memcpy(vals, S->vals.data(), S->vals.size() * sizeof(uint32_t));
  if (ranges) std::memcpy(ranges, S->ranges.data(), S->ranges.size() * sizeof(int32_t));
}

// Per-Gaussian projection results.
//   f64 [n, 13]: u, v, conic a, b, c, opacity, r, rgb[3], depth(FP64), Sigma2 A, C
//   f32 [n, 4] : depth32, u32, v32, r32
//   i32 [n, 9] : valid, visible, tx0, tx1, ty0, ty1, rect_amb, grad_amb, pad
//   i32 [n, 4] : union rectangle atx0, atx1, aty0, aty1
void or_get_records(void* h, double* f64, float* f32, int32_t* i32, int32_t* arect) {
  State* S = (State*)h;
  for (int64_t i = 0; i < S->sc.n; ++i) {
    const Rec& g = S->rec[i];
    if (f64) {
      double* o = f64 + 13 * i;
      double vals[13] = {g.u, g.v, g.a, g.b, g.c, g.o, g.r, g.rgb[0], g.rgb[1], g.rgb[2], g.p[2], g.A, g.C};
      if (!g.valid) for (double& x : vals) x = 0;
      std::memcpy(o, vals, sizeof vals);
    }
    if (f32) { f32[4 * i] = g.depth32; f32[4 * i + 1] = g.u32; f32[4 * i + 2] = g.v32; f32[4 * i + 3] = g.r32; }
    if (i32) {
      int32_t* o = i32 + 9 * i;
      o[0] = g.valid; o[1] = g.visible; o[2] = g.tx0; o[3] = g.tx1; o[4] = g.ty0; o[5] = g.ty1;
      o[6] = g.rect_amb; o[7] = g.grad_amb; o[8] = 0;
    }
    if (arect) { arect[4 * i] = g.atx0; arect[4 * i + 1] = g.atx1; arect[4 * i + 2] = g.aty0; arect[4 * i + 3] = g.aty1; }
  }
}

// Directional central differences of L = sum over channels and pixels of w[c, p] * I[c, p], one
// Gaussian at a time (the adjoint's pin at memory scale).  Target k is Gaussian ids[k] of the
// rendered state; its raw parameters move by +-eps * dirs[k] (dirs [m, F], F = 11 + 3K: mean 3,
// log-scale 3, quaternion 4, logit 1, SH 3K, the layout of the raw parameters).  Only that Gaussian
// is projected again and only the tiles of its rectangle are composited again: every other pixel
// is unchanged by construction, so the difference of the two partial sums is the difference of
// the full loss.  out[k] = (L(+) - L(-)) / (2 eps).  flags[k] = 1 when the perturbation changes a
// decision (validity, tile rectangle, the Gaussian's position in any of its tile lists, a guard-band
// or colour-clamp side, or any skip / clamp / stop decision of an affected pixel); a flagged sample
// crosses a discontinuity and is not a derivative.  Runs targets in parallel.
void or_fd_directional(void* h, const double* w, int64_t m, const int64_t* ids, const double* dirs, double eps,
                       double* out, int32_t* flags) {
  State* S = (State*)h;
  const int K = S->K, F = 11 + 3 * K;
  const int W = S->cam.width, H = S->cam.height, TS = S->op.tile;
  const size_t plane = (size_t)W * H;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t k = 0; k < m; ++k) {
    const int64_t id = ids[k];
    const Rec& g0 = S->rec[id];
    out[k] = 0.0;
    flags[k] = 0;
    if (!g0.visible) { flags[k] = 1; continue; }
    // composite the Gaussian's tiles with record `rec` for it; returns the partial loss and the
    // decision hash of those pixels
    auto partial = [&](const Rec* rec, uint64_t* hh) {
      double L = 0.0;
      int64_t ev = 0, bl = 0;
      *hh = 0;
      for (int ty = g0.ty0; ty <= g0.ty1; ++ty)
        for (int tx = g0.tx0; tx <= g0.tx1; ++tx) {
          const int t = ty * S->tiles_x + tx;
          for (int y = ty * TS; y < std::min(H, (ty + 1) * TS); ++y)
            for (int x = tx * TS; x < std::min(W, (tx + 1) * TS); ++x) {
              double C[3], T;
              int32_t last;
              bool amb = false;
              render_pixel(*S, x, y, t, C, &T, &last, &amb, &ev, &bl, hh, nullptr, rec, (uint32_t)id);
              const size_t p = (size_t)y * W + x;
              for (int ch = 0; ch < 3; ++ch) L += w[ch * plane + p] * (C[ch] + T * S->op.bg[ch]);
            }
        }
      return L;
    };
    uint64_t h0 = 0;
    partial(nullptr, &h0);
    double Ls[2];
    for (int sgn = 0; sgn < 2 && !flags[k]; ++sgn) {
      const double e = sgn == 0 ? eps : -eps;
      const double* d = dirs + (size_t)k * F;
      std::vector<double> means(3), ls(3), q(4), lg(1), sh(3 * (size_t)K);
      for (int c = 0; c < 3; ++c) means[c] = S->sc.means[3 * id + c] + e * d[c];
      for (int c = 0; c < 3; ++c) ls[c] = S->sc.log_scales[3 * id + c] + e * d[3 + c];
      for (int c = 0; c < 4; ++c) q[c] = S->sc.quats[4 * id + c] + e * d[6 + c];
      lg[0] = S->sc.logits[id] + e * d[10];
      for (int c = 0; c < 3 * K; ++c) sh[c] = S->sc.sh[(size_t)id * 3 * K + c] + e * d[11 + c];
      State one;
      one.sc = S->sc;
      one.sc.n = 1;
      one.sc.means = means.data(); one.sc.log_scales = ls.data(); one.sc.quats = q.data();
      one.sc.logits = lg.data(); one.sc.sh = sh.data();
      one.cam = S->cam;
      one.op = S->op;
      one.K = K;
      one.tiles_x = S->tiles_x;
      one.tiles_y = S->tiles_y;
      one.rec.assign(1, Rec());
      project(one, 0);
      const Rec& g1 = one.rec[0];
      bool same = g1.valid && g1.visible && g1.tx0 == g0.tx0 && g1.tx1 == g0.tx1 && g1.ty0 == g0.ty0 &&
                  g1.ty1 == g0.ty1 && g1.clx == g0.clx && g1.cly == g0.cly;
      for (int ch = 0; ch < 3 && same; ++ch) same = (g1.pre[ch] > 0) == (g0.pre[ch] > 0);
      // the new key keeps the Gaussian's place in every list it is in
      for (int ty = g0.ty0; ty <= g0.ty1 && same; ++ty)
        for (int tx = g0.tx0; tx <= g0.tx1 && same; ++tx) {
          const int t = ty * S->tiles_x + tx;
          const int32_t s0 = S->ranges[2 * t], s1 = S->ranges[2 * t + 1];
          int32_t j = s0;
          while (j < s1 && S->vals[j] != (uint32_t)id) ++j;
          if (j == s1) { same = false; break; }
          const uint64_t key = ((uint64_t)t << 32) | float_bits(g1.depth32);
          if (j > s0 && !(S->keys[j - 1] < key || (S->keys[j - 1] == key && S->vals[j - 1] < (uint32_t)id))) same = false;
          if (j + 1 < s1 && !(key < S->keys[j + 1] || (key == S->keys[j + 1] && (uint32_t)id < S->vals[j + 1]))) same = false;
        }
      if (!same) { flags[k] = 1; break; }
      uint64_t h1 = 0;
      Ls[sgn] = partial(&g1, &h1);
      if (h1 != h0) flags[k] = 1;
    }
    if (!flags[k]) out[k] = (Ls[0] - Ls[1]) / (2.0 * eps);
  }
}

// Transmittance after each blended Gaussian of one pixel, front to back; returns the count.
int32_t or_pixel_trace(void* h, int x, int y, double* T_after, uint32_t* gauss, int32_t cap) {
  State* S = (State*)h;
  int TS = S->op.tile;
  int t = (y / TS) * S->tiles_x + x / TS;
  std::vector<Step> tr;
  double C[3], T;
  int32_t last;
  bool amb;
  int64_t e = 0, b = 0;
  uint64_t hh = 0;
  render_pixel(*S, x, y, t, C, &T, &last, &amb, &e, &b, &hh, &tr);
  int32_t n = 0;
  for (auto& s : tr) {
    if (n >= cap) break;
    T_after[n] = s.Tb * (1.0 - s.alpha);
    gauss[n] = s.g;
    ++n;
  }
  return (int32_t)tr.size();
}

// Adjoint of the forward pass.  dL_dimg [3,H,W].  Outputs (overwritten, zeros for culled):
// g_means [n,3], g_log_scales [n,3], g_quats [n,4], g_logits [n], g_sh [n,K,3], and optionally
// g2d [n,9] = dL/d(u, v, conic a, b, c, opacity, r, g, b) and g2d_abs [n], the densification
// statistic: the sum over pixels of |dL/du| + |dL/dv| of each pixel's own contribution (the
// per-pixel terms of g2d's first two columns, taken in absolute value before summing).
void or_backward(void* h, const double* dL_dimg, double* g_means, double* g_log_scales, double* g_quats,
                 double* g_logits, double* g_sh, double* g2d_out, double* g2d_abs_out) {
  State* S = (State*)h;
  const OrOpts& op = S->op;
  const OrCamera& cm = S->cam;
  int W = cm.width, H = cm.height, TS = op.tile;
  int64_t n = S->sc.n;
  int K = S->K;
  int tiles = S->tiles_x * S->tiles_y;
  std::vector<double> g2d(9 * (size_t)n, 0.0), g2d_abs((size_t)n, 0.0);
  // per-tile partial sums (the nine g2d fields, then the absolute-value statistic), merged
  // serially for a deterministic result
  std::vector<std::vector<std::pair<uint32_t, std::array<double, 10>>>> parts(tiles);
#pragma omp parallel for schedule(dynamic, 1)
  for (int t = 0; t < tiles; ++t) {
    if (!S->rendered_tile[t]) continue;
    int tx = t % S->tiles_x, ty = t / S->tiles_x;
    std::vector<std::array<double, 10>> acc;
    std::vector<uint32_t> ids;
    int32_t s0 = S->ranges[2 * t];
    int32_t len = S->ranges[2 * t + 1] - s0;
    acc.assign(len, std::array<double, 10>{});
    for (int y = ty * TS; y < std::min(H, (ty + 1) * TS); ++y)
      for (int x = tx * TS; x < std::min(W, (tx + 1) * TS); ++x) {
        std::vector<Step> tr;
        double C[3], T;
        int32_t last;
        bool amb;
        int64_t e = 0, b = 0;
        uint64_t hh = 0;
        render_pixel(*S, x, y, t, C, &T, &last, &amb, &e, &b, &hh, &tr);
        size_t p = (size_t)y * W + x;
        double gp[3] = {dL_dimg[p], dL_dimg[(size_t)W * H + p], dL_dimg[2 * (size_t)W * H + p]};
        double Acc[3] = {T * op.bg[0], T * op.bg[1], T * op.bg[2]};   // colour behind
        for (int k = (int)tr.size() - 1; k >= 0; --k) {
          const Step& s = tr[k];
          const Rec& g = S->rec[s.g];
          auto& a = acc[s.pos];
          double dl_da = 0;
          for (int ch = 0; ch < 3; ++ch) {
            a[6 + ch] += s.alpha * s.Tb * gp[ch];
            dl_da += s.Tb * g.rgb[ch] * gp[ch] - Acc[ch] * gp[ch] / (1.0 - s.alpha);
          }
          for (int ch = 0; ch < 3; ++ch) Acc[ch] += g.rgb[ch] * s.alpha * s.Tb;
          if (s.clamped) continue;
          a[5] += dl_da * s.G;
          double dl_dpow = dl_da * s.alpha;
          double dx = x - g.u, dy = y - g.v;
          const double du = dl_dpow * (g.a * dx + g.b * dy), dv = dl_dpow * (g.b * dx + g.c * dy);
          a[0] += du;
          a[1] += dv;
          a[9] += std::fabs(du) + std::fabs(dv);
          a[2] += dl_dpow * (-0.5 * dx * dx);
          a[3] += dl_dpow * (-dx * dy);
          a[4] += dl_dpow * (-0.5 * dy * dy);
        }
      }
    for (int32_t j = 0; j < len; ++j) parts[t].push_back({S->vals[s0 + j], acc[j]});
  }
  for (int t = 0; t < tiles; ++t)
    for (auto& pr : parts[t]) {
      for (int f = 0; f < 9; ++f) g2d[9 * (size_t)pr.first + f] += pr.second[f];
      g2d_abs[pr.first] += pr.second[9];
    }
  if (g2d_out) std::memcpy(g2d_out, g2d.data(), g2d.size() * sizeof(double));
  if (g2d_abs_out) std::memcpy(g2d_abs_out, g2d_abs.data(), g2d_abs.size() * sizeof(double));

  // chain rule per Gaussian
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    const Rec& g = S->rec[i];
    double* gm = g_means + 3 * i;
    double* gs = g_log_scales + 3 * i;
    double* gq = g_quats + 4 * i;
    double* gsh = g_sh + (size_t)i * K * 3;
    std::fill(gm, gm + 3, 0.0); std::fill(gs, gs + 3, 0.0); std::fill(gq, gq + 4, 0.0);
    g_logits[i] = 0.0;
    std::fill(gsh, gsh + 3 * K, 0.0);
    if (!g.visible) continue;
    const double* d2 = &g2d[9 * (size_t)i];
    // opacity
    g_logits[i] = d2[5] * g.o * (1.0 - g.o);
    // colour
    double Y[16], dY[16][3];
    sh_basis(S->sc.sh_degree, g.d, Y, dY);
    double dd[3] = {0, 0, 0};
    for (int ch = 0; ch < 3; ++ch) {
      double dpre = g.pre[ch] > 0 ? d2[6 + ch] : 0.0;
      for (int k = 0; k < K; ++k) {
        gsh[3 * k + ch] = dpre * Y[k];
        double coef = S->sc.sh[((size_t)i * K + k) * 3 + ch];
        for (int c = 0; c < 3; ++c) dd[c] += dpre * coef * dY[k][c];
      }
    }
    double dotd = g.d[0] * dd[0] + g.d[1] * dd[1] + g.d[2] * dd[2];
    for (int c = 0; c < 3; ++c) gm[c] += (dd[c] - g.d[c] * dotd) / g.dirlen;
    // conic -> 2D covariance:  dSigma2 = -Q G Q with Q = conic matrix, G = dL/dQ (sym.)
    double Q[4] = {g.a, g.b, g.b, g.c};
    double G[4] = {d2[2], 0.5 * d2[3], 0.5 * d2[3], d2[4]};
    double QG[4], dS2[4];
    matmul(Q, G, QG, 2, 2, 2);
    matmul(QG, Q, dS2, 2, 2, 2);
    for (double& x : dS2) x = -x;
    // Sigma2 = T Sigma T^T + dil I, T = J W
    double T[6], Tt[6], tmp[6], dSigma[9], dT[6], dJ[6], Wt[9];
    matmul(g.J, g.W, T, 2, 3, 3);
    transpose(T, Tt, 2, 3);
    matmul(Tt, dS2, tmp, 3, 2, 2);          // 3x2
    matmul(tmp, T, dSigma, 3, 2, 3);        // 3x3
    double dS2T[6];
    matmul(dS2, T, dS2T, 2, 2, 3);
    matmul(dS2T, g.Sigma, dT, 2, 3, 3);
    for (double& x : dT) x *= 2.0;
    transpose(g.W, Wt, 3, 3);
    matmul(dT, Wt, dJ, 2, 3, 3);
    // J -> view-space position
    double z = g.p[2], x = g.p[0], y = g.p[1];
    double fx = cm.fx, fy = cm.fy;
    double dp[3] = {0, 0, 0};
    double xzc = g.clx ? (x / z > 0 ? 1 : -1) * op.guard * 0.5 * cm.width / fx : x / z;
    double yzc = g.cly ? (y / z > 0 ? 1 : -1) * op.guard * 0.5 * cm.height / fy : y / z;
    dp[2] += dJ[0] * (-fx / (z * z)) + dJ[4] * (-fy / (z * z));
    // J02 = -fx * xzc / z
    double dJ02_dz = fx * xzc / (z * z) - (g.clx ? 0.0 : fx / z * (-x / (z * z)));
    double dJ02_dx = g.clx ? 0.0 : -fx / (z * z);
    double dJ12_dz = fy * yzc / (z * z) - (g.cly ? 0.0 : fy / z * (-y / (z * z)));
    double dJ12_dy = g.cly ? 0.0 : -fy / (z * z);
    dp[0] += dJ[2] * dJ02_dx;
    dp[2] += dJ[2] * dJ02_dz;
    dp[1] += dJ[5] * dJ12_dy;
    dp[2] += dJ[5] * dJ12_dz;
    // pixel position
    dp[0] += d2[0] * fx / z;
    dp[2] += d2[0] * (-fx * x / (z * z));
    dp[1] += d2[1] * fy / z;
    dp[2] += d2[1] * (-fy * y / (z * z));
    for (int c = 0; c < 3; ++c) gm[c] += g.W[c] * dp[0] + g.W[3 + c] * dp[1] + g.W[6 + c] * dp[2];
    // Sigma = M M^T, M = Rq diag(s)
    double M[9], dM[9];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) M[3 * r + c] = g.Rq[3 * r + c] * g.s[c];
    matmul(dSigma, M, dM, 3, 3, 3);
    for (double& v : dM) v *= 2.0;
    double dRq[9];
    for (int c = 0; c < 3; ++c) {
      double ds = 0;
      for (int r = 0; r < 3; ++r) { ds += dM[3 * r + c] * g.Rq[3 * r + c]; dRq[3 * r + c] = dM[3 * r + c] * g.s[c]; }
      gs[c] = ds * g.s[c];
    }
    double pR[4][9];
    quat_to_rot_partials(g.qn, pR);
    double dqn[4];
    for (int k = 0; k < 4; ++k) { dqn[k] = 0; for (int e = 0; e < 9; ++e) dqn[k] += dRq[e] * pR[k][e]; }
    double dot = 0;
    for (int k = 0; k < 4; ++k) dot += g.qn[k] * dqn[k];
    for (int k = 0; k < 4; ++k) gq[k] = (dqn[k] - g.qn[k] * dot) / g.qnorm;
  }
}

// ---------------------------------------------------------------------------------------------
// Loss, Eq. 1: L = (1 - lambda) mean|x - y| + lambda (1 - mean SSIM(x, y)), with its gradient
// with respect to the rendered image x.  Images are [3, H, W]; SSIM uses an 11x11 Gaussian
// window (sigma 1.5, normalised), zero padding, C1 = 0.01^2, C2 = 0.03^2.
//   S = (2 mx my + C1)(2 sxy + C2) / ((mx^2 + my^2 + C1)(sx^2 + sy^2 + C2))
// where m = w*x, sx^2 = w*(x^2) - mx^2, sxy = w*(x y) - mx my.
// ---------------------------------------------------------------------------------------------
void gauss_window(double* w11) {
  double s = 0;
  for (int i = 0; i < 11; ++i) { w11[i] = std::exp(-((i - 5) * (i - 5)) / (2.0 * 1.5 * 1.5)); s += w11[i]; }
  for (int i = 0; i < 11; ++i) w11[i] /= s;
}

// 2D window correlation with zero padding (the window is symmetric, so this is also its
// convolution and its own adjoint).
void conv2(const double* in, double* out, int H, int W, const double* w) {
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      double s = 0;
      for (int j = -5; j <= 5; ++j) {
        int yy = y + j;
        if (yy < 0 || yy >= H) continue;
        for (int i = -5; i <= 5; ++i) {
          int xx = x + i;
          if (xx < 0 || xx >= W) continue;
          s += w[j + 5] * w[i + 5] * in[(size_t)yy * W + xx];
        }
      }
      out[(size_t)y * W + x] = s;
    }
}

double or_ssim_map(const double* x, const double* y, int H, int W, double* smap /*optional [3,H,W]*/) {
  double w[11];
  gauss_window(w);
  size_t P = (size_t)H * W;
  std::vector<double> xx(P), yy(P), xy(P), mx(P), my(P), exx(P), eyy(P), exy(P);
  double total = 0;
  const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
  for (int ch = 0; ch < 3; ++ch) {
    const double* X = x + ch * P;
    const double* Y = y + ch * P;
    for (size_t p = 0; p < P; ++p) { xx[p] = X[p] * X[p]; yy[p] = Y[p] * Y[p]; xy[p] = X[p] * Y[p]; }
    conv2(X, mx.data(), H, W, w); conv2(Y, my.data(), H, W, w);
    conv2(xx.data(), exx.data(), H, W, w); conv2(yy.data(), eyy.data(), H, W, w); conv2(xy.data(), exy.data(), H, W, w);
    for (size_t p = 0; p < P; ++p) {
      double sx = exx[p] - mx[p] * mx[p], sy = eyy[p] - my[p] * my[p], sxy = exy[p] - mx[p] * my[p];
      double s = (2 * mx[p] * my[p] + C1) * (2 * sxy + C2) / ((mx[p] * mx[p] + my[p] * my[p] + C1) * (sx + sy + C2));
      if (smap) smap[ch * P + p] = s;
      total += s;
    }
  }
  return total / (3.0 * P);
}

double or_loss_l1_dssim(const double* x, const double* y, int H, int W, double lambda, double* grad /*[3,H,W] or null*/) {
  double w[11];
  gauss_window(w);
  size_t P = (size_t)H * W;
  double inv = 1.0 / (3.0 * P);
  const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
  double l1 = 0, ssim = 0;
  std::vector<double> xx(P), yy(P), xy(P), mx(P), my(P), exx(P), eyy(P), exy(P), ga(P), gb(P), gc(P), ca(P), cb(P), cc(P);
  for (int ch = 0; ch < 3; ++ch) {
    const double* X = x + ch * P;
    const double* Y = y + ch * P;
    for (size_t p = 0; p < P; ++p) {
      double d = X[p] - Y[p];
      l1 += std::fabs(d);
      if (grad) grad[ch * P + p] = (1.0 - lambda) * inv * (d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0));
      xx[p] = X[p] * X[p]; yy[p] = Y[p] * Y[p]; xy[p] = X[p] * Y[p];
    }
    conv2(X, mx.data(), H, W, w); conv2(Y, my.data(), H, W, w);
    conv2(xx.data(), exx.data(), H, W, w); conv2(yy.data(), eyy.data(), H, W, w); conv2(xy.data(), exy.data(), H, W, w);
    for (size_t p = 0; p < P; ++p) {
      double m1 = mx[p], m2 = my[p];
      double sx = exx[p] - m1 * m1, sy = eyy[p] - m2 * m2, sxy = exy[p] - m1 * m2;
      double N1 = 2 * m1 * m2 + C1, N2 = 2 * sxy + C2, D1 = m1 * m1 + m2 * m2 + C1, D2 = sx + sy + C2;
      double s = N1 * N2 / (D1 * D2);
      ssim += s;
      // dS with respect to the raw moments mx, exx, exy of x
      double dS_dmx = (2 * m2 * N2 + N1 * (-2 * m2)) / (D1 * D2) - s * (2 * m1 / D1 + (-2 * m1) / D2);
      double dS_dexx = -s / D2;
      double dS_dexy = 2 * N1 / (D1 * D2);
      double G = -lambda * inv;   // dL/dS(p)
      ga[p] = G * dS_dmx; gb[p] = G * dS_dexx; gc[p] = G * dS_dexy;
    }
    if (grad) {
      conv2(ga.data(), ca.data(), H, W, w); conv2(gb.data(), cb.data(), H, W, w); conv2(gc.data(), cc.data(), H, W, w);
      for (size_t p = 0; p < P; ++p) grad[ch * P + p] += ca[p] + 2.0 * X[p] * cb[p] + Y[p] * cc[p];
    }
  }
  return (1.0 - lambda) * l1 * inv + lambda * (1.0 - ssim * inv);
}

}  // extern "C"
