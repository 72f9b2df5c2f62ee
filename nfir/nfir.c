/* NFIR mass-spring-damper trajectory simulator (synthetic input data; no GP arithmetic).
 *
 * Three unit masses in a chain wall-m1-m2-m3 (free end). Each link carries a spring force
 * k*d + 0.5*d^3 (k = 1) and a damper 0.2*d' in parallel, d being the link's relative displacement.
 * A piecewise-constant force u ~ U[-1, 1], held for 20 samples, acts on m1. RK4 with dt = 0.01
 * from rest, one sample every 10 steps. Sample i records the force u_i applied during interval i
 * and y_i = q3 at the end of that interval plus N(0, 0.01^2) noise.
 * Random numbers: SplitMix64 (Steele, Lea, Flood 2014), 53-bit uniforms, Box-Muller normals.
 * Built with -ffp-contract=off so no multiply-add is fused behind the code's back.
 */
#include <math.h>
#include <stdint.h>

static uint64_t sm64_next(uint64_t* s) {
  uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static double sm64_uniform(uint64_t* s) { return (double)(sm64_next(s) >> 11) * (1.0 / 9007199254740992.0); }
static double sm64_normal(uint64_t* s) {
  double u1 = 1.0 - sm64_uniform(s); /* (0, 1] */
  double u2 = sm64_uniform(s);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

void nfir_splitmix64(uint64_t seed, int64_t count, uint64_t* out) {
  uint64_t s = seed;
  for (int64_t i = 0; i < count; ++i) out[i] = sm64_next(&s);
}

static void accel(const double* q, const double* v, double u, double* a) {
  const double k = 1.0, c3 = 0.5, c = 0.2;
  double d1 = q[0], d2 = q[1] - q[0], d3 = q[2] - q[1];
  double e1 = v[0], e2 = v[1] - v[0], e3 = v[2] - v[1];
  double f1 = k * d1 + c3 * d1 * d1 * d1 + c * e1;
  double f2 = k * d2 + c3 * d2 * d2 * d2 + c * e2;
  double f3 = k * d3 + c3 * d3 * d3 * d3 + c * e3;
  a[0] = u - f1 + f2; /* unit masses */
  a[1] = f3 - f2;
  a[2] = -f3;
}

/* Simulates n_samples samples from seed; writes u_out[i], y_out[i]. */
void nfir_simulate(int64_t n_samples, uint64_t seed, double* u_out, double* y_out) {
  const double h = 0.01;
  uint64_t s = seed;
  double q[3] = {0, 0, 0}, v[3] = {0, 0, 0}, u = 0.0;
  for (int64_t i = 0; i < n_samples; ++i) {
    if (i % 20 == 0) u = 2.0 * sm64_uniform(&s) - 1.0;
    for (int st = 0; st < 10; ++st) {
      double a1[3], a2[3], a3[3], a4[3], qt[3], vt[3], v2[3], v3[3];
      accel(q, v, u, a1);
      for (int j = 0; j < 3; ++j) { qt[j] = q[j] + 0.5 * h * v[j]; vt[j] = v[j] + 0.5 * h * a1[j]; }
      for (int j = 0; j < 3; ++j) v2[j] = vt[j];
      accel(qt, vt, u, a2);
      for (int j = 0; j < 3; ++j) { qt[j] = q[j] + 0.5 * h * v2[j]; vt[j] = v[j] + 0.5 * h * a2[j]; }
      for (int j = 0; j < 3; ++j) v3[j] = vt[j];
      accel(qt, vt, u, a3);
      for (int j = 0; j < 3; ++j) { qt[j] = q[j] + h * v3[j]; vt[j] = v[j] + h * a3[j]; }
      accel(qt, vt, u, a4);
      for (int j = 0; j < 3; ++j) {
        q[j] += h / 6.0 * (v[j] + 2.0 * v2[j] + 2.0 * v3[j] + vt[j]);
        v[j] += h / 6.0 * (a1[j] + 2.0 * a2[j] + 2.0 * a3[j] + a4[j]);
      }
    }
    u_out[i] = u;
    y_out[i] = q[2] + 0.01 * sm64_normal(&s);
  }
}
