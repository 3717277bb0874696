/*
 * dvnr_oracle.c -- plain, slow, FP64 CPU oracle of the DVNR hot path.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, by __graft_entry__.smoke() and
 * by the CPU-baseline leg of bench.py. The product library never uses it.
 * It shares no code, header, table or constant generator with the CUDA path.
 *
 * Paper: "Distributed Neural Representation for Reactive In Situ
 * Visualization" (arXiv 2304.10516). Hash encoding: Mueller et al. 2022
 * (cited by the paper in Sec. 3 for the encoding layer). Philox-4x32-10:
 * Salmon et al. 2011, "Parallel random numbers: as easy as 1, 2, 3".
 *
 * Arithmetic is FP64 throughout, except where the mixed-precision path is
 * emulated (mixed != 0): there values are rounded to IEEE binary16 at the
 * same points where the GPU stores FP16 operands. Compile with
 * -ffp-contract=off so that a*b+c is never fused.
 */
#define _GNU_SOURCE
#include "dvnr_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define FIX_ONE (1LL << 24) /* coordinates are 24-bit fixed point: u = m / 2^24 */

int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the parallel loops from now on (n >= 1); returns the number in
 * effect afterwards. Timing only: results do not depend on it beyond the
 * order of FP64 additions in the batch sums.                               */
int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Configuration. Level resolution N_l = floor(N_min * b^l) (Mueller et al.,
 * Eq. 2-3; the DVNR paper defers to that paper in Sec. 3). A level is stored
 * densely when its (N_l+1)^3 vertices fit in T, otherwise hashed into T
 * entries (Mueller et al. Sec. 3; DVNR Sec. 3.4 speaks of "dense" and
 * "hashed" levels).                                                         */
int orc_cfg_init(orc_cfg* c, int32_t L, int32_t F, int32_t log2T,
                 int32_t base_res, double growth, int32_t width,
                 int32_t n_hidden) {
  memset(c, 0, sizeof(*c));
  if (L < 1 || L > ORC_MAX_LEVELS) return -1;
  if (!(F == 1 || F == 2 || F == 4 || F == 8)) return -1;
  if (log2T < 4 || log2T > 24) return -1;
  if (base_res < 1 || !(growth >= 1.0)) return -1;
  if (width < 1 || width > 256 || n_hidden < 1 || n_hidden > ORC_MAX_HIDDEN)
    return -1;
  c->L = L; c->F = F; c->log2T = log2T; c->base_res = base_res;
  c->growth = growth; c->width = width; c->n_hidden = n_hidden;
  c->in_dim = L * F;
  const int64_t T = 1LL << log2T;
  int64_t off = 0;
  for (int l = 0; l < L; ++l) {
    double r = floor((double)base_res * pow(growth, (double)l));
    if (r > (double)(1 << 21)) return -1;
    int64_t N = (int64_t)r;
    c->N[l] = (int32_t)N;
    int64_t verts = (N + 1) * (N + 1) * (N + 1);
    c->dense[l] = verts <= T;
    c->entries[l] = c->dense[l] ? verts : T;
    c->offset[l] = off;
    off += c->entries[l] * F;
  }
  c->n_enc = off;
  int64_t w = c->n_enc;
  c->w_off[0] = w;
  w += (int64_t)width * c->in_dim;
  for (int k = 1; k < n_hidden; ++k) {
    c->w_off[k] = w;
    w += (int64_t)width * width;
  }
  c->w_off[n_hidden] = w; /* output row w_out */
  w += width;
  c->n_params = w;
  c->n_mlp = w - c->n_enc;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Philox-4x32-10 (Salmon et al. 2011): ten rounds of two 32x32->64 bit
 * multiplications with the round constants 0xD2511F53 / 0xCD9E8D57 and the
 * Weyl key increments 0x9E3779B9 / 0xBB67AE85.                             */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)0xD2511F53u * x0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;
    uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
    uint32_t y1 = (uint32_t)p1;
    uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
    uint32_t y3 = (uint32_t)p0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* IEEE-754 binary16 round-to-nearest-even of a double (the FP16 storage of
 * the mixed-precision path, Sec. 3.4 stores weights as 16-bit floats).     */
double orc_round_half(double x) {
  if (isnan(x) || isinf(x)) return x;
  double a = fabs(x);
  if (a >= 65520.0) return copysign(INFINITY, x);
  double q;
  if (a < 6.103515625e-05) { /* subnormal range: quantum 2^-24 */
    q = nearbyint(a * 16777216.0) / 16777216.0;
  } else {
    int e;
    frexp(a, &e); /* a = f * 2^e, f in [0.5, 1): 11 significant bits */
    double quantum = ldexp(1.0, e - 11);
    q = nearbyint(a / quantum) * quantum;
  }
  return copysign(q, x);
}

/* ------------------------------------------------------------------------ */
/* Vertex -> table index. Dense: x + y(N+1) + z(N+1)^2. Hashed: the spatial
 * hash of Mueller et al. (Eq. 4), XOR of the coordinates times the primes
 * 1, 2654435761, 805459861, modulo 2^32, then modulo T.                    */
uint32_t orc_corner_index(const orc_cfg* c, int level, int64_t x, int64_t y,
                          int64_t z) {
  int64_t N1 = (int64_t)c->N[level] + 1;
  if (c->dense[level]) return (uint32_t)(x + y * N1 + z * N1 * N1);
  uint32_t h = ((uint32_t)x * 1u) ^ ((uint32_t)y * 2654435761u) ^
               ((uint32_t)z * 805459861u);
  return h & (uint32_t)((1u << c->log2T) - 1u);
}

/* ------------------------------------------------------------------------ */
/* Initialisation (the paper is silent). Tables U(-1e-4, 1e-4) as in
 * Mueller et al.; MLP Glorot-uniform +-sqrt(6/(fan_in+fan_out)). The uniform
 * is u = (r0 >> 8) 2^-24 from Philox(ctr = {i_lo, i_hi, 0, 'INIT'},
 * key = seed); value = lo + (hi - lo) u in FP64, then rounded to binary32
 * (the GPU keeps FP32 master weights).                                     */
void orc_init_params(const orc_cfg* c, uint64_t seed, double* theta) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int64_t i = 0; i < c->n_params; ++i) {
    uint32_t ctr[4] = {(uint32_t)i, (uint32_t)((uint64_t)i >> 32), 0u,
                       0x494E4954u};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    double u = (double)(r[0] >> 8) / 16777216.0;
    double lo, hi;
    if (i < c->n_enc) {
      lo = -1e-4;
      hi = 1e-4;
    } else {
      int64_t fan_in, fan_out;
      if (i >= c->w_off[c->n_hidden]) {
        fan_in = c->width; fan_out = 1;
      } else if (i < c->w_off[0] + (int64_t)c->width * c->in_dim) {
        fan_in = c->in_dim; fan_out = c->width;
      } else {
        fan_in = c->width; fan_out = c->width;
      }
      double limit = sqrt(6.0 / (double)(fan_in + fan_out));
      lo = -limit;
      hi = limit;
    }
    double span = hi - lo;
    double v = lo + span * u;
    theta[i] = (double)(float)v;
  }
}

/* ------------------------------------------------------------------------ */
/* Boundary sampling (Sec. 3.3, Eq. 2): an equal-weight mixture of the six
 * half-Gaussians centred on the faces of [0,1]^3. A half-normal offset is
 * drawn by inverse-CDF sampling through a 4096-segment piecewise-linear
 * quantile table q(p) = sigma * sqrt(2) * erfinv(p), stored as 24-bit fixed
 * point (the last knot is q(1 - 2^-24)). Here erfinv is found by bisection
 * on the C library's erf().                                                */
static double erfinv_bisect(double p) {
  double a = 0.0, b = 8.0;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (a + b);
    if (mid == a || mid == b) break;
    if (erf(mid) < p) a = mid; else b = mid;
  }
  return 0.5 * (a + b);
}

void orc_quantile_table(double sigma, int64_t* tab) {
  for (int k = 0; k <= ORC_QTAB; ++k) {
    double p = (k < ORC_QTAB) ? (double)k / ORC_QTAB : 1.0 - ldexp(1.0, -24);
    double x = (k == 0) ? 0.0 : erfinv_bisect(p);
    double q = sigma * (1.41421356237309504880 * x);
    tab[k] = llround(q * (double)FIX_ONE);
  }
}

/* One batch of training coordinates (Sec. 3.2 uniform sampling and Sec. 3.3
 * boundary sampling; the first floor(lambda*B) samples are boundary samples,
 * the rest uniform, so that every step draws exactly B samples).
 * Philox counter {i, iter, model, 'SAM' + attempt}, key = seed.
 *   uniform : m_a = r_a >> 8 for a = x, y, z.
 *   boundary: face = floor(6 r0 / 2^32) -> axis = face/2, side = face%2;
 *             offset from the quantile table at u = r1 >> 8; the coordinate
 *             on that axis is offset (side 0) or 2^24 - offset (side 1);
 *             the two other axes take r2 >> 8, r3 >> 8 in axis order.
 *             An offset beyond 1 is redrawn with attempt + 1 (at most 255
 *             times, then clamped).
 * Returns the number of redraws.                                           */
int orc_sample(uint64_t seed, uint32_t model, uint64_t iter, int32_t batch,
               double lambda_bnd, const int64_t* qtab, uint32_t* m_out) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  const int64_t nb = (int64_t)floor(lambda_bnd * (double)batch);
  int redraws = 0;
  for (int64_t i = 0; i < batch; ++i) {
    uint32_t* m = m_out + 3 * i;
    if (i >= nb) {
      uint32_t ctr[4] = {(uint32_t)i, (uint32_t)iter, model, 0x53414D00u};
      uint32_t r[4];
      orc_philox4x32_10(ctr, key, r);
      m[0] = r[0] >> 8; m[1] = r[1] >> 8; m[2] = r[2] >> 8;
      continue;
    }
    for (uint32_t attempt = 0;; ++attempt) {
      uint32_t ctr[4] = {(uint32_t)i, (uint32_t)iter, model,
                         0x53414D00u + attempt};
      uint32_t r[4];
      orc_philox4x32_10(ctr, key, r);
      uint32_t face = (uint32_t)(((uint64_t)r[0] * 6u) >> 32);
      uint32_t axis = face >> 1, side = face & 1u;
      uint32_t u24 = r[1] >> 8;
      uint32_t k = u24 >> 12, fr = u24 & 4095u;
      int64_t off = qtab[k] + (((qtab[k + 1] - qtab[k]) * (int64_t)fr) >> 12);
      if (off > FIX_ONE && attempt < 255) {
        ++redraws;
        continue;
      }
      if (off > FIX_ONE) off = FIX_ONE;
      uint32_t other[2] = {r[2] >> 8, r[3] >> 8};
      int o = 0;
      for (uint32_t a = 0; a < 3; ++a) {
        if (a == axis)
          m[a] = side ? (uint32_t)(FIX_ONE - off) : (uint32_t)off;
        else
          m[a] = other[o++];
      }
      break;
    }
  }
  return redraws;
}

/* Position of a fixed-point coordinate on a lattice of n cells:
 * p = m * n / 2^24, base = min(floor(p), n - 1), frac = p - base.          */
static void lattice(uint32_t m, int64_t n, int64_t* base, double* frac) {
  int64_t p = (int64_t)m * n;
  int64_t b = p >> 24;
  if (b > n - 1) b = n - 1;
  if (b < 0) b = 0;
  *base = b;
  *frac = (double)(p - (b << 24)) / (double)FIX_ONE;
}

/* Target lookup (Sec. 3.2: trilinear interpolation of the ground truth at
 * the sampled coordinate). The stored block of n voxels per axis spans
 * [0,1] from the first to the last voxel centre: position u (n - 1).       */
double orc_volume_trilinear(const float* vol, int64_t nx, int64_t ny,
                            int64_t nz, const uint32_t m[3]) {
  int64_t n[3] = {nx, ny, nz}, b[3];
  double f[3];
  for (int a = 0; a < 3; ++a) {
    if (n[a] < 2) { b[a] = 0; f[a] = 0.0; continue; }
    lattice(m[a], n[a] - 1, &b[a], &f[a]);
  }
  double v = 0.0;
  for (int c = 0; c < 8; ++c) {
    int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
    double w = (cx ? f[0] : 1.0 - f[0]) * (cy ? f[1] : 1.0 - f[1]) *
               (cz ? f[2] : 1.0 - f[2]);
    int64_t x = b[0] + (n[0] > 1 ? cx : 0);
    int64_t y = b[1] + (n[1] > 1 ? cy : 0);
    int64_t z = b[2] + (n[2] > 1 ? cz : 0);
    v += w * (double)vol[(z * ny + y) * nx + x];
  }
  return v;
}

/* ------------------------------------------------------------------------ */
/* Multiresolution hash encoding, forward (Sec. 3 / Mueller et al. Sec. 3):
 * per level, the 8 vertices of the enclosing cell, their trilinear weights
 * and the F features of each, interpolated and concatenated level-major.
 * Position p = u N_l with no half-cell offset (reading: the paper is silent;
 * u = 1 uses the last cell with frac = 1).                                 */
typedef struct {
  uint32_t idx[8];
  double w[8];
} corner_set;

static void level_corners(const orc_cfg* c, int l, const uint32_t m[3],
                          corner_set* cs) {
  int64_t b[3];
  double f[3];
  for (int a = 0; a < 3; ++a) lattice(m[a], c->N[l], &b[a], &f[a]);
  for (int k = 0; k < 8; ++k) {
    int cx = k & 1, cy = (k >> 1) & 1, cz = (k >> 2) & 1;
    cs->w[k] = (cx ? f[0] : 1.0 - f[0]) * (cy ? f[1] : 1.0 - f[1]) *
               (cz ? f[2] : 1.0 - f[2]);
    cs->idx[k] = orc_corner_index(c, l, b[0] + cx, b[1] + cy, b[2] + cz);
  }
}

/* round_params: round each table value to binary16 when it is read;
 * round_acts: round the interpolated feature to binary16. The public entry
 * rounds both in mixed mode; the batch paths pre-round the parameters once. */
static void encode_impl(const orc_cfg* c, const double* theta, const uint32_t m[3],
                        int round_params, int round_acts, double* x0) {
  for (int l = 0; l < c->L; ++l) {
    corner_set cs;
    level_corners(c, l, m, &cs);
    for (int f = 0; f < c->F; ++f) {
      double acc = 0.0;
      for (int k = 0; k < 8; ++k) {
        double v = theta[c->offset[l] + (int64_t)cs.idx[k] * c->F + f];
        if (round_params) v = orc_round_half(v);
        acc += cs.w[k] * v;
      }
      x0[l * c->F + f] = round_acts ? orc_round_half(acc) : acc;
    }
  }
}

void orc_encode(const orc_cfg* c, const double* theta, const uint32_t m[3],
                int mixed, double* x0) {
  encode_impl(c, theta, m, mixed, mixed, x0);
}

/* Parameters as the mixed-precision path stores them: every value rounded to
 * binary16 once (returns theta itself when not mixed; free with
 * release_params). */
static const double* prepare_params(const orc_cfg* c, const double* theta, int mixed) {
  if (!mixed) return theta;
  double* r = (double*)malloc(sizeof(double) * (size_t)c->n_params);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t i = 0; i < c->n_params; ++i) r[i] = orc_round_half(theta[i]);
  return r;
}
static void release_params(const double* prepared, const double* theta) {
  if (prepared != theta) free((void*)prepared);
}

void orc_encode_batch(const orc_cfg* c, const double* theta, int64_t n,
                      const uint32_t* m, int mixed, double* x0) {
  const double* th = prepare_params(c, theta, mixed);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t i = 0; i < n; ++i) encode_impl(c, th, m + 3 * i, 0, mixed, x0 + i * c->in_dim);
  release_params(th, theta);
}

/* Normalised targets (v - min)/(max - min) at n fixed-point coordinates
 * (Sec. 3.1: values normalised to [0,1] by the partition's min and max).   */
void orc_targets(const float* vol, int64_t nx, int64_t ny, int64_t nz,
                 int64_t n, const uint32_t* m, double vmin, double vmax,
                 double* out) {
  const double range = vmax - vmin;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t i = 0; i < n; ++i) {
    double v = orc_volume_trilinear(vol, nx, ny, nz, m + 3 * i);
    out[i] = range > 0.0 ? (v - vmin) / range : 0.0;
  }
}

/* ------------------------------------------------------------------------ */
/* Forward and backward of one batch (Sec. 3: encoding + ReLU MLP, no output
 * activation and no biases -- reading: the paper's backend, tiny-cuda-nn's
 * fully fused MLP, has none; Sec. 3.3: unweighted L1 over the mixed batch).
 *
 *   loss      0: L1 = mean |y - t|, dL/dy = sign(y - t)/B, sign(0) = 0
 *             1: L2 = mean (y - t)^2, dL/dy = 2 (y - t)/B
 *   mixed     emulate the FP16 rounding points of the mixed-precision path
 *             (tables, weights, encoding output, hidden activations, scaled
 *             output gradient and hidden-layer gradients are binary16)
 *   loss_scale S: the output gradient is multiplied by S before the
 *             backward pass and every accumulated gradient divided by S
 *   grad_norm_count  B in dL/dy (normally n)
 *   flip      optional n x (H*width + 1) bytes: 1 inverts the derivative
 *             decision of that ReLU unit (z > 0) or, in the last slot, the
 *             sign of the L1 derivative. Used by the tests to bound what a
 *             branch taken differently at a kink can change.
 *   grad_enc  += table gradients (n_enc), may be NULL
 *   grad_mlp  += weight gradients (n_mlp), may be NULL
 *   y_out, dx0_out (n x in_dim, unscaled), margin_out: optional per sample;
 *             margin = min(|z| over hidden units, |y - t| for L1)
 *   zabs_out  optional n x (H*width + 1): |z| of every hidden unit and, in
 *             the last slot, |y - t| (L1) or +inf (L2)
 * Returns the mean loss.                                                    */
typedef struct {
  double* h;   /* (H+1) x maxw activations, h[0] = x0 */
  double* z;   /* (H+1) x width pre-activations       */
  double* dz;  /* width                               */
  double* dh;  /* maxw                                */
} scratch_t;

static double sample_fwd_bwd(const orc_cfg* c, const double* theta,
                             const uint32_t m[3], double target, int32_t loss,
                             int32_t mixed, double S, double inv_B,
                             const uint8_t* flip, double* gmlp, double* dx0,
                             double* y_out, double* margin, double* zabs, scratch_t* s) {
  const int W = c->width, H = c->n_hidden, D = c->in_dim;
  const int maxw = W > D ? W : D;
  double* h = s->h;
  double* z = s->z;
#define HROW(k) (h + (int64_t)(k) * maxw)
#define ZROW(k) (z + (int64_t)(k) * W)
#define WGT(v) (v) /* parameters arrive pre-rounded in mixed mode */
  encode_impl(c, theta, m, 0, mixed, HROW(0));
  double mg = INFINITY;
  for (int k = 0; k < H; ++k) {
    const int in = k == 0 ? D : W;
    const double* Wk = theta + c->w_off[k];
    for (int j = 0; j < W; ++j) {
      double acc = 0.0;
      for (int i = 0; i < in; ++i) acc += WGT(Wk[(int64_t)j * in + i]) * HROW(k)[i];
      ZROW(k + 1)[j] = acc;
      double r = acc > 0.0 ? acc : 0.0;
      HROW(k + 1)[j] = mixed ? orc_round_half(r) : r;
      if (fabs(acc) < mg) mg = fabs(acc);
      if (zabs) zabs[k * W + j] = fabs(acc);
    }
  }
  const double* wout = theta + c->w_off[H];
  double y = 0.0;
  for (int j = 0; j < W; ++j) y += WGT(wout[j]) * HROW(H)[j];
  const double d = y - target;
  double lval, g;
  if (loss == 0) {
    lval = fabs(d);
    g = d > 0.0 ? 1.0 : (d < 0.0 ? -1.0 : 0.0);
    if (flip && flip[H * W]) g = (g == 0.0) ? 1.0 : -g;
    if (fabs(d) < mg) mg = fabs(d);
    if (zabs) zabs[H * W] = fabs(d);
  } else {
    lval = d * d;
    g = 2.0 * d;
    if (zabs) zabs[H * W] = INFINITY;
  }
  if (y_out) *y_out = y;
  if (margin) *margin = mg;
  const double gy = g * S * inv_B; /* scaled dL/dy */
  const double inv_S = 1.0 / S;
  double* dz = s->dz;
  double* dh = s->dh;
  /* output layer */
  const double gy_op = mixed ? orc_round_half(gy) : gy;
  if (gmlp)
    for (int j = 0; j < W; ++j)
      gmlp[c->w_off[H] - c->n_enc + j] += gy_op * HROW(H)[j] * inv_S;
  for (int j = 0; j < W; ++j) {
    int on = ZROW(H)[j] > 0.0;
    if (flip && flip[(H - 1) * W + j]) on = !on;
    double v = on ? gy * WGT(wout[j]) : 0.0;
    dz[j] = mixed ? orc_round_half(v) : v;
  }
  /* hidden layers, top down */
  for (int k = H - 1; k >= 0; --k) {
    const int in = k == 0 ? D : W;
    const double* Wk = theta + c->w_off[k];
    if (gmlp) {
      double* gk = gmlp + (c->w_off[k] - c->n_enc);
      for (int j = 0; j < W; ++j)
        for (int i = 0; i < in; ++i)
          gk[(int64_t)j * in + i] += dz[j] * HROW(k)[i] * inv_S;
    }
    for (int i = 0; i < in; ++i) {
      double acc = 0.0;
      for (int j = 0; j < W; ++j) acc += WGT(Wk[(int64_t)j * in + i]) * dz[j];
      dh[i] = acc;
    }
    if (k == 0) {
      for (int i = 0; i < D; ++i) dx0[i] = dh[i] * inv_S;
    } else {
      for (int i = 0; i < W; ++i) {
        int on = ZROW(k)[i] > 0.0;
        if (flip && flip[(k - 1) * W + i]) on = !on;
        double v = on ? dh[i] : 0.0;
        dz[i] = mixed ? orc_round_half(v) : v;
      }
    }
  }
#undef HROW
#undef ZROW
#undef WGT
  return lval;
}

double orc_fwd_bwd(const orc_cfg* c, const double* theta, int64_t n,
                   const uint32_t* m, const double* target, int32_t loss,
                   int32_t mixed, double loss_scale, int64_t grad_norm_count,
                   const uint8_t* flip, double* grad_enc, double* grad_mlp,
                   double* y_out, double* dx0_out, double* margin_out,
                   double* zabs_out) {
  const int D = c->in_dim, W = c->width, H = c->n_hidden;
  const int maxw = W > D ? W : D;
  const int64_t nunits = (int64_t)H * W + 1;
  const double inv_B = 1.0 / (double)grad_norm_count;
  double* dx0_all = dx0_out ? dx0_out : (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * D);
  const int nt = orc_threads();
  double* gpart = NULL;
  if (grad_mlp) gpart = (double*)calloc((size_t)nt * c->n_mlp, sizeof(double));
  double loss_sum = 0.0;
  const double* th = prepare_params(c, theta, mixed);
#ifdef _OPENMP
#pragma omp parallel reduction(+ : loss_sum)
#endif
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    scratch_t s;
    s.h = (double*)malloc(sizeof(double) * (size_t)(H + 1) * maxw);
    s.z = (double*)malloc(sizeof(double) * (size_t)(H + 1) * W);
    s.dz = (double*)malloc(sizeof(double) * (size_t)W);
    s.dh = (double*)malloc(sizeof(double) * (size_t)maxw);
    double* gmine = gpart ? gpart + (int64_t)tid * c->n_mlp : NULL;
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
    for (int64_t i = 0; i < n; ++i) {
      loss_sum += sample_fwd_bwd(
          c, th, m + 3 * i, target[i], loss, mixed, loss_scale, inv_B,
          flip ? flip + i * nunits : NULL, gmine, dx0_all + i * D,
          y_out ? y_out + i : NULL, margin_out ? margin_out + i : NULL,
          zabs_out ? zabs_out + i * nunits : NULL, &s);
    }
    free(s.h); free(s.z); free(s.dz); free(s.dh);
  }
  release_params(th, theta);
  if (grad_mlp) {
    for (int t = 0; t < nt; ++t)
      for (int64_t p = 0; p < c->n_mlp; ++p) grad_mlp[p] += gpart[(int64_t)t * c->n_mlp + p];
    free(gpart);
  }
  /* encoding backward: scatter dL/dx0 times the trilinear weights */
  if (grad_enc) {
    for (int64_t i = 0; i < n; ++i) {
      for (int l = 0; l < c->L; ++l) {
        corner_set cs;
        level_corners(c, l, m + 3 * i, &cs);
        for (int k = 0; k < 8; ++k)
          for (int f = 0; f < c->F; ++f)
            grad_enc[c->offset[l] + (int64_t)cs.idx[k] * c->F + f] +=
                cs.w[k] * dx0_all[i * D + l * c->F + f];
      }
    }
  }
  if (!dx0_out) free(dx0_all);
  return loss_sum * inv_B;
}

/* ------------------------------------------------------------------------ */
/* Adam (Sec. 3.6: beta1 = 0.9, beta2 = 0.999, eps = 1e-8, L2 weight decay
 * 1e-9 added to the gradient of every parameter -- reading: the paper does
 * not say which parameters decay; constant learning rate). Kingma & Ba
 * bias correction with eps added to sqrt(v_hat). A step with a non-finite
 * gradient is skipped; in mixed precision it also halves the loss scale,
 * and growth_interval finite steps in a row double it.                     */
void orc_adam(const orc_cfg* c, const orc_train_cfg* tc, orc_state* st,
              double* theta, double* mom1, double* mom2, const double* grad) {
  int finite = 1;
  for (int64_t i = 0; i < c->n_params; ++i)
    if (!isfinite(grad[i])) { finite = 0; break; }
  if (!finite) {
    st->skipped += 1;
    st->good_steps = 0;
    if (tc->mixed) st->loss_scale *= 0.5;
    return;
  }
  st->adam_t += 1;
  const double t = (double)st->adam_t;
  const double bc1 = 1.0 - pow(tc->beta1, t);
  const double bc2 = 1.0 - pow(tc->beta2, t);
  for (int64_t i = 0; i < c->n_params; ++i) {
    double g = grad[i] + tc->weight_decay * theta[i];
    mom1[i] = tc->beta1 * mom1[i] + (1.0 - tc->beta1) * g;
    mom2[i] = tc->beta2 * mom2[i] + (1.0 - tc->beta2) * g * g;
    double mh = mom1[i] / bc1;
    double vh = mom2[i] / bc2;
    theta[i] -= tc->lr * mh / (sqrt(vh) + tc->eps);
  }
  if (tc->mixed) {
    st->good_steps += 1;
    if (st->good_steps >= tc->growth_interval) {
      st->loss_scale *= 2.0;
      st->good_steps = 0;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Training loop (Sec. 3.2): per iteration sample B coordinates, look up
 * their targets by trilinear interpolation of the min/max-normalised volume
 * (Sec. 3.1 / 3.2 normalise values to [0,1] by the partition's min and max,
 * ghost layer included), forward, loss, backward, Adam.                    */
double orc_train(const orc_cfg* c, const orc_train_cfg* tc, orc_state* st,
                 double* theta, double* mom1, double* mom2, const float* vol,
                 int64_t nx, int64_t ny, int64_t nz, double vmin, double vmax,
                 int64_t steps, double* loss_hist) {
  const int32_t B = tc->batch;
  int64_t qtab[ORC_QTAB + 1];
  orc_quantile_table(tc->sigma_bnd, qtab);
  uint32_t* m = (uint32_t*)malloc(sizeof(uint32_t) * 3 * (size_t)B);
  double* tgt = (double*)malloc(sizeof(double) * (size_t)B);
  double* grad = (double*)malloc(sizeof(double) * (size_t)c->n_params);
  const double range = vmax - vmin;
  double last = 0.0;
  for (int64_t s = 0; s < steps; ++s) {
    orc_sample(tc->seed, tc->model, (uint64_t)st->iter, B, tc->lambda_bnd, qtab, m);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < B; ++i) {
      double v = orc_volume_trilinear(vol, nx, ny, nz, m + 3 * i);
      tgt[i] = range > 0.0 ? (v - vmin) / range : 0.0;
    }
    memset(grad, 0, sizeof(double) * (size_t)c->n_params);
    const double S = tc->mixed ? st->loss_scale : 1.0;
    last = orc_fwd_bwd(c, theta, B, m, tgt, tc->loss, tc->mixed, S, B, NULL,
                       grad, grad + c->n_enc, NULL, NULL, NULL, NULL);
    if (loss_hist) loss_hist[s] = last;
    orc_adam(c, tc, st, theta, mom1, mom2, grad);
    st->iter += 1;
  }
  free(m); free(tgt); free(grad);
  return last;
}

/* ------------------------------------------------------------------------ */
/* Iteration budget and early stop (Sec. 3.2). The paper makes the number of
 * iterations proportional to the partition's voxel count, N_train^max =
 * max(N_train^min, ceil(N_vox / N_batch) N_epoch), and lets training end
 * once a moving average of the loss is below a user threshold. Readings
 * (the paper is silent): N_vox counts the owned voxels (no ghost layer); the
 * moving average is exponential with factor d, started at the first finite
 * loss of the call; steps whose gradient was non-finite (skipped by Adam)
 * count against the budget but not in the average; the test follows every
 * step's update, so a call that stops after step t has applied t steps.   */
int64_t orc_max_iterations(int64_t n_vox, int64_t batch, int64_t steps,
                           int64_t epochs, int64_t min_steps) {
  int64_t n = steps;
  if (epochs > 0) n = ((n_vox + batch - 1) / batch) * epochs;
  return n > min_steps ? n : min_steps;
}

/* Sec. 3.2 scales the hash table with the partition's share of the voxels,
 * printed as T = max(T_min, T_ref ceil(N_vox / N_vox^global)); the ceiling
 * of a share <= 1 is 1, so read literally T would never change. Reading: the
 * ceiling applies to the product, rounded up to the power of two that a hash
 * table size must be. Found by doubling from 1 in exact integer arithmetic
 * (2^k N_vox^global >= T_ref N_vox). R_0 = floor(R_ref cbrt(T / T_ref)),
 * taken from the FP64 cube root and corrected to the exact floor when R_ref
 * is an integer (R^3 T_ref <= R_ref^3 T).                                     */
void orc_adaptive_encoding(int64_t n_vox, int64_t n_vox_global, int32_t log2_T_ref,
                           int32_t log2_T_min, double R_ref, int32_t* log2_T,
                           int32_t* base_res) {
  /* smallest k with 2^k n_global >= 2^log2_T_ref n_vox, in long double to
   * keep the products exact up to 2^63 */
  int32_t k = 0;
  const long double need = ldexpl((long double)n_vox, log2_T_ref);
  while (ldexpl((long double)n_vox_global, k) < need) ++k;
  if (k < log2_T_min) k = log2_T_min;
  *log2_T = k;
  const double ratio = ldexp(1.0, k - log2_T_ref);
  double r = floor(R_ref * cbrt(ratio));
  if (R_ref == floor(R_ref)) {
    /* exact floor for integer R_ref: largest R with R^3 <= R_ref^3 ratio */
    const long double lim = (long double)R_ref * R_ref * R_ref * (long double)ratio;
    while (r > 0 && (long double)r * r * r > lim) r -= 1.0;
    while ((long double)(r + 1) * (r + 1) * (r + 1) <= lim) r += 1.0;
  }
  *base_res = r < 1.0 ? 1 : (int32_t)r;
}

int64_t orc_stop_step(const double* losses, const int32_t* finite, int64_t n,
                      double decay, double stop_loss, double* ema_out) {
  double m = -1.0;
  int have = 0;
  int64_t t = 0;
  while (t < n) {
    const double L = losses[t];
    const int ok = finite ? finite[t] != 0 : 1;
    t += 1;
    if (!ok) continue;
    m = have ? decay * m + (1.0 - decay) * L : L;
    have = 1;
    if (stop_loss > 0.0 && m < stop_loss) break;
  }
  if (ema_out) *ema_out = m;
  return t;
}

int64_t orc_train_budget(const orc_cfg* c, const orc_train_cfg* tc, orc_state* st,
                         double* theta, double* mom1, double* mom2, const float* vol,
                         int64_t nx, int64_t ny, int64_t nz, double vmin, double vmax,
                         int64_t budget, double stop_loss, double decay,
                         double* loss_hist, double* ema_out, int32_t* stopped_out) {
  double m = -1.0;
  int have = 0, stopped = 0;
  int64_t t = 0;
  while (t < budget && !stopped) {
    const int64_t skipped_before = st->skipped;
    const double L = orc_train(c, tc, st, theta, mom1, mom2, vol, nx, ny, nz, vmin, vmax, 1, NULL);
    if (loss_hist) loss_hist[t] = L;
    t += 1;
    if (st->skipped != skipped_before) continue;  /* non-finite step */
    m = have ? decay * m + (1.0 - decay) * L : L;
    have = 1;
    if (stop_loss > 0.0 && m < stop_loss) stopped = 1;
  }
  if (ema_out) *ema_out = m;
  if (stopped_out) *stopped_out = stopped;
  return t;
}

/* ------------------------------------------------------------------------ */
/* Inference (Sec. 3: "the neural network can output v on-demand for any
 * arbitrary coordinates", decoded value y (max - min) + min, Sec. 4.1 keeps
 * the value range). No clamp of y (reading: the paper is silent).          */
void orc_decode_unit(const orc_cfg* c, const double* theta, int64_t n,
                     const uint32_t* m, int mixed, double vmin, double vmax,
                     double* out) {
  const double* th = prepare_params(c, theta, mixed);
#ifdef _OPENMP
#pragma omp parallel
#endif
  {
    const int W = c->width, H = c->n_hidden, D = c->in_dim;
    const int maxw = W > D ? W : D;
    double* a = (double*)malloc(sizeof(double) * (size_t)maxw);
    double* b = (double*)malloc(sizeof(double) * (size_t)maxw);
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
    for (int64_t s = 0; s < n; ++s) {
      encode_impl(c, th, m + 3 * s, 0, mixed, a);
      for (int k = 0; k < H; ++k) {
        const int in = k == 0 ? D : W;
        const double* Wk = th + c->w_off[k];
        for (int j = 0; j < W; ++j) {
          double acc = 0.0;
          for (int i = 0; i < in; ++i) {
            double w = Wk[(int64_t)j * in + i];
            acc += w * a[i];
          }
          double r = acc > 0.0 ? acc : 0.0;
          b[j] = mixed ? orc_round_half(r) : r;
        }
        double* t = a; a = b; b = t;
      }
      const double* wout = th + c->w_off[H];
      double y = 0.0;
      for (int j = 0; j < W; ++j) y += wout[j] * a[j];
      out[s] = y * (vmax - vmin) + vmin;
    }
    free(a); free(b);
  }
  release_params(th, theta);
}

/* Stored voxel j of n -> fixed-point coordinate round(j 2^24 / (n - 1)),
 * computed exactly in integers (the INR domain [0,1] spans the first to the
 * last stored voxel centre, ghost layer included; Sec. 3.3 and Fig. 3A).    */
uint32_t orc_grid_coord(int64_t j, int64_t n) {
  if (n < 2) return 0;
  return (uint32_t)((2 * j * FIX_ONE + (n - 1)) / (2 * (n - 1)));
}

/* Decode back to the grid (Sec. 3 and Sec. 4.1): the owned voxels of the
 * block (the ghost layer stripped), x fastest.                             */
void orc_decode_grid(const orc_cfg* c, const double* theta, const int64_t n[3],
                     int32_t ghost, int mixed, double vmin, double vmax,
                     double* out) {
  const int64_t ex = n[0] - 2 * ghost, ey = n[1] - 2 * ghost, ez = n[2] - 2 * ghost;
  const int64_t cnt = ex * ey * ez;
  uint32_t* m = (uint32_t*)malloc(sizeof(uint32_t) * 3 * (size_t)cnt);
  for (int64_t z = 0; z < ez; ++z)
    for (int64_t y = 0; y < ey; ++y)
      for (int64_t x = 0; x < ex; ++x) {
        int64_t i = (z * ey + y) * ex + x;
        m[3 * i + 0] = orc_grid_coord(x + ghost, n[0]);
        m[3 * i + 1] = orc_grid_coord(y + ghost, n[1]);
        m[3 * i + 2] = orc_grid_coord(z + ghost, n[2]);
      }
  orc_decode_unit(c, theta, cnt, m, mixed, vmin, vmax, out);
  free(m);
}

/* ------------------------------------------------------------------------ */
/* Direct volume rendering of decoded blocks (Sec. 4.3; the paper gives no
 * camera or transfer function, so these are readings): orthographic view
 * along +z over the union of the owned boxes, one ray per pixel centre,
 * spr samples at the centres of spr equal steps in z, trilinear on each
 * block's own decoded grid (clamped at its edge), linear transfer function
 * rgb = c0 + (c1 - c0) v, alpha = alpha_max v with v normalised by
 * [v_lo, v_hi] and clamped to [0,1], front-to-back compositing without
 * early termination (sort-last order = block order along +z).
 * tf = {r0, g0, b0, r1, g1, b1, alpha_max, v_lo, v_hi}.                     */
void orc_render(int32_t n_blocks, const double* const* grids,
                const int64_t* lo, const int64_t* hi, const double* tf,
                int32_t w, int32_t h, int32_t spr, double* rgba) {
  double LO[3], HI[3];
  for (int a = 0; a < 3; ++a) {
    LO[a] = 1e300; HI[a] = -1e300;
    for (int b = 0; b < n_blocks; ++b) {
      if ((double)lo[3 * b + a] < LO[a]) LO[a] = (double)lo[3 * b + a];
      if ((double)hi[3 * b + a] > HI[a]) HI[a] = (double)hi[3 * b + a];
    }
  }
  const double vlo = tf[7], vhi = tf[8];
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t pix = 0; pix < (int64_t)w * h; ++pix) {
    const int px = (int)(pix % w), py = (int)(pix / w);
    const double X = LO[0] - 0.5 + (px + 0.5) * (HI[0] - LO[0]) / w;
    const double Y = LO[1] - 0.5 + (py + 0.5) * (HI[1] - LO[1]) / h;
    double C[3] = {0, 0, 0}, A = 0.0;
    for (int k = 0; k < spr; ++k) {
      const double Z = LO[2] - 0.5 + (k + 0.5) * (HI[2] - LO[2]) / spr;
      const double P[3] = {X, Y, Z};
      int blk = -1;
      for (int b = 0; b < n_blocks && blk < 0; ++b) {
        int in = 1;
        for (int a = 0; a < 3; ++a)
          if (!(P[a] >= lo[3 * b + a] - 0.5 && P[a] < hi[3 * b + a] - 0.5)) in = 0;
        if (in) blk = b;
      }
      if (blk < 0) continue;
      int64_t e[3], base[3];
      double fr[3];
      for (int a = 0; a < 3; ++a) {
        e[a] = hi[3 * blk + a] - lo[3 * blk + a];
        double q = P[a] - (double)lo[3 * blk + a];
        if (q < 0.0) q = 0.0;
        if (q > (double)(e[a] - 1)) q = (double)(e[a] - 1);
        int64_t bq = (int64_t)floor(q);
        if (bq > e[a] - 2) bq = e[a] - 2;
        if (bq < 0) bq = 0;
        base[a] = bq;
        fr[a] = e[a] > 1 ? q - (double)bq : 0.0;
      }
      const double* g = grids[blk];
      double v = 0.0;
      for (int cc = 0; cc < 8; ++cc) {
        int cx = cc & 1, cy = (cc >> 1) & 1, cz = (cc >> 2) & 1;
        double wgt = (cx ? fr[0] : 1 - fr[0]) * (cy ? fr[1] : 1 - fr[1]) *
                     (cz ? fr[2] : 1 - fr[2]);
        int64_t x = base[0] + (e[0] > 1 ? cx : 0);
        int64_t y = base[1] + (e[1] > 1 ? cy : 0);
        int64_t z = base[2] + (e[2] > 1 ? cz : 0);
        v += wgt * g[(z * e[1] + y) * e[0] + x];
      }
      double vn = (vhi > vlo) ? (v - vlo) / (vhi - vlo) : 0.0;
      if (vn < 0.0) vn = 0.0;
      if (vn > 1.0) vn = 1.0;
      const double alpha = tf[6] * vn;
      for (int ch = 0; ch < 3; ++ch) {
        const double col = tf[ch] + (tf[3 + ch] - tf[ch]) * vn;
        C[ch] += (1.0 - A) * alpha * col;
      }
      A += (1.0 - A) * alpha;
    }
    rgba[4 * pix + 0] = C[0];
    rgba[4 * pix + 1] = C[1];
    rgba[4 * pix + 2] = C[2];
    rgba[4 * pix + 3] = A;
  }
}

/* Direct volume rendering from the networks (Sec. 4.3: the paper's renderer
 * infers the models at the ray samples instead of decoding grids). The same
 * readings as orc_render for the camera, samples, block ownership, transfer
 * function and front-to-back compositing; a sample's value is its block's
 * network at the sample position. The position maps into the block's unit
 * domain as in point decoding: u = (P - (lo - ghost)) / (n_stored - 1),
 * clamped to [0, 1] and rounded to the nearest multiple of 2^-24. Samples
 * are first assigned and collected per block, each block's network is
 * evaluated once over its samples, then every ray is composited in order. */
void orc_render_inr(const orc_cfg* c, int32_t n_blocks, const double* const* thetas,
                    const int64_t* lo, const int64_t* hi, const int32_t* ghost,
                    int mixed, const double* vmin, const double* vmax,
                    const double* tf, int32_t w, int32_t h, int32_t spr,
                    int64_t n_pix, const int64_t* pix, double* rgba) {
  double LO[3], HI[3];
  for (int a = 0; a < 3; ++a) {
    LO[a] = 1e300; HI[a] = -1e300;
    for (int b = 0; b < n_blocks; ++b) {
      if ((double)lo[3 * b + a] < LO[a]) LO[a] = (double)lo[3 * b + a];
      if ((double)hi[3 * b + a] > HI[a]) HI[a] = (double)hi[3 * b + a];
    }
  }
  const int64_t ns = n_pix * (int64_t)spr;
  int32_t* owner = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ns > 0 ? ns : 1));
  uint32_t* m = (uint32_t*)malloc(sizeof(uint32_t) * 3 * (size_t)(ns > 0 ? ns : 1));
  double* val = (double*)calloc((size_t)(ns > 0 ? ns : 1), sizeof(double));
  /* 1: block and unit-lattice coordinate of every sample */
  for (int64_t i = 0; i < n_pix; ++i) {
    const int px = (int)(pix[i] % w), py = (int)(pix[i] / w);
    const double X = LO[0] - 0.5 + (px + 0.5) * (HI[0] - LO[0]) / w;
    const double Y = LO[1] - 0.5 + (py + 0.5) * (HI[1] - LO[1]) / h;
    for (int k = 0; k < spr; ++k) {
      const int64_t q = i * spr + k;
      const double Z = LO[2] - 0.5 + (k + 0.5) * (HI[2] - LO[2]) / spr;
      const double P[3] = {X, Y, Z};
      int blk = -1;
      for (int b = 0; b < n_blocks && blk < 0; ++b) {
        int in = 1;
        for (int a = 0; a < 3; ++a)
          if (!(P[a] >= lo[3 * b + a] - 0.5 && P[a] < hi[3 * b + a] - 0.5)) in = 0;
        if (in) blk = b;
      }
      owner[q] = blk;
      if (blk < 0) continue;
      for (int a = 0; a < 3; ++a) {
        const int64_t n_st = hi[3 * blk + a] - lo[3 * blk + a] + 2 * (int64_t)ghost[blk];
        double u = 0.0;
        if (n_st > 1) {
          u = (P[a] - (double)(lo[3 * blk + a] - ghost[blk])) / (double)(n_st - 1);
          if (u < 0.0) u = 0.0;
          if (u > 1.0) u = 1.0;
        }
        m[3 * q + a] = (uint32_t)nearbyint(u * 16777216.0);
      }
    }
  }
  /* 2: each block's network over its samples */
  for (int b = 0; b < n_blocks; ++b) {
    int64_t cnt = 0;
    for (int64_t q = 0; q < ns; ++q) cnt += owner[q] == b;
    if (cnt == 0) continue;
    uint32_t* mb = (uint32_t*)malloc(sizeof(uint32_t) * 3 * (size_t)cnt);
    double* vb = (double*)malloc(sizeof(double) * (size_t)cnt);
    int64_t j = 0;
    for (int64_t q = 0; q < ns; ++q)
      if (owner[q] == b) {
        mb[3 * j] = m[3 * q]; mb[3 * j + 1] = m[3 * q + 1]; mb[3 * j + 2] = m[3 * q + 2];
        ++j;
      }
    orc_decode_unit(c, thetas[b], cnt, mb, mixed, vmin[b], vmax[b], vb);
    j = 0;
    for (int64_t q = 0; q < ns; ++q)
      if (owner[q] == b) val[q] = vb[j++];
    free(mb); free(vb);
  }
  /* 3: front-to-back compositing of every ray */
  const double vlo = tf[7], vhi = tf[8];
  for (int64_t i = 0; i < n_pix; ++i) {
    double C[3] = {0, 0, 0}, A = 0.0;
    for (int k = 0; k < spr; ++k) {
      const int64_t q = i * spr + k;
      if (owner[q] < 0) continue;
      double vn = (vhi > vlo) ? (val[q] - vlo) / (vhi - vlo) : 0.0;
      if (vn < 0.0) vn = 0.0;
      if (vn > 1.0) vn = 1.0;
      const double alpha = tf[6] * vn;
      for (int ch = 0; ch < 3; ++ch) C[ch] += (1.0 - A) * alpha * (tf[ch] + (tf[3 + ch] - tf[ch]) * vn);
      A += (1.0 - A) * alpha;
    }
    rgba[4 * i] = C[0]; rgba[4 * i + 1] = C[1]; rgba[4 * i + 2] = C[2]; rgba[4 * i + 3] = A;
  }
  free(owner); free(m); free(val);
}

/* Reconstruction error in FP64 (Sec. 5: PSNR from the mean squared error;
 * max-abs error is reported beside it).                                     */
double orc_mse(const double* a, const float* b, int64_t n, double* max_abs) {
  double s = 0.0, mx = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double d = a[i] - (double)b[i];
    s += d * d;
    if (fabs(d) > mx) mx = fabs(d);
  }
  if (max_abs) *max_abs = mx;
  return n > 0 ? s / (double)n : 0.0;
}
