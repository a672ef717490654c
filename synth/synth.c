/*
 * Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.
 *
 * This file generates INPUT DATA only: scalar fields shaped like the paper's
 * datasets (Table 2), threshold masks, uniform sample coordinates, initial
 * parameter values and the training targets sampled from a voxel field.  It
 * contains none of the F-Hash method's arithmetic (no level schedule, no F-Hash
 * row mapping, no quadrilinear embedding interpolation, no MLP, no Adam, no ray
 * marching); the method lives in the CUDA library and, separately, in the oracle.
 *
 * Random numbers come from SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014), used as a
 * counter-based generator: value i of stream s under seed k is the i-th output
 * of SplitMix64 seeded with key(k, s), where key(k, s) is itself the s-th output
 * of SplitMix64 seeded with k.
 *
 * Build: gcc -O2 -fopenmp -fPIC -shared -ffp-contract=off (no fast-math), so that
 * x86 and Arm hosts give the same bits except where libm's exp/tanh differ.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* i-th output (0-based) of SplitMix64 whose state starts at `seed`. */
uint64_t synth_splitmix64_at(uint64_t seed, uint64_t i) { return mix64(seed + (i + 1) * GOLDEN); }

static inline uint64_t stream_key(uint64_t seed, uint64_t stream) { return synth_splitmix64_at(seed, stream); }
static inline uint64_t rnd64(uint64_t key, uint64_t i) { return mix64(key + (i + 1) * GOLDEN); }
/* Uniform in [0,1): top 24 bits, exact in float and double. */
static inline double unit24(uint64_t x) { return (double)(x >> 40) * (1.0 / 16777216.0); }

/* out[i] = (float)(lo + (hi - lo) * U_i), U_i = unit24 of value offset+i of (seed, stream). */
void synth_uniform(uint64_t seed, uint64_t stream, uint64_t offset, int64_t n, double lo, double hi, float* out) {
    uint64_t key = stream_key(seed, stream);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) out[i] = (float)(lo + (hi - lo) * unit24(rnd64(key, offset + (uint64_t)i)));
}

/* ---------------------------------------------------------------- value noise */
/* Lattice of values U(-1,1) with spacing (sx voxels, st steps), quadrilinear between lattice points.
 * Lattice dims: ceil(n/s)+2 per axis; lattice value index = linear index over those dims. */
typedef struct { int64_t lx, ly, lz, lt; double sx, st; float* v; } noise_lattice;

static void lattice_init(noise_lattice* L, uint64_t seed, uint64_t stream, int64_t nx, int64_t ny, int64_t nz,
                         int64_t nt, double sx, double st) {
    L->sx = sx; L->st = st;
    L->lx = (int64_t)ceil(nx / sx) + 2; L->ly = (int64_t)ceil(ny / sx) + 2; L->lz = (int64_t)ceil(nz / sx) + 2;
    L->lt = (int64_t)ceil(nt / st) + 2;
    int64_t n = L->lx * L->ly * L->lz * L->lt;
    L->v = (float*)malloc((size_t)n * sizeof(float));
    synth_uniform(seed, stream, 0, n, -1.0, 1.0, L->v);
}

/* Trilinear lattice slice at time step t (time-lerped once per step). */
static float* lattice_slice(const noise_lattice* L, int64_t t) {
    double pt = t / L->st; int64_t it = (int64_t)floor(pt); double ft = pt - it;
    int64_t n3 = L->lx * L->ly * L->lz;
    float* s = (float*)malloc((size_t)n3 * sizeof(float));
    const float* a = L->v + it * n3; const float* b = a + n3;
    for (int64_t i = 0; i < n3; ++i) s[i] = (float)((1.0 - ft) * a[i] + ft * b[i]);
    return s;
}

static inline double slice_eval(const noise_lattice* L, const float* s, int64_t x, int64_t y, int64_t z) {
    double px = x / L->sx, py = y / L->sx, pz = z / L->sx;
    int64_t ix = (int64_t)floor(px), iy = (int64_t)floor(py), iz = (int64_t)floor(pz);
    double fx = px - ix, fy = py - iy, fz = pz - iz;
    const float* b = s + (iz * L->ly + iy) * L->lx + ix;
    int64_t sy = L->lx, sz = L->lx * L->ly;
    double c00 = b[0] * (1 - fx) + b[1] * fx, c10 = b[sy] * (1 - fx) + b[sy + 1] * fx;
    double c01 = b[sz] * (1 - fx) + b[sz + 1] * fx, c11 = b[sz + sy] * (1 - fx) + b[sz + sy + 1] * fx;
    double c0 = c00 * (1 - fy) + c10 * fy, c1 = c01 * (1 - fy) + c11 * fy;
    return c0 * (1 - fz) + c1 * fz;
}

/* ---------------------------------------------------------------- fields */
/*
 * kind 1: Gaussian blobs on straight lines (the 32^3 x 8 instance): 4 blobs, sigma 3, amplitude 1,
 *         centres U[8,24]^3, unit directions uniform on the sphere, 1 voxel/step, plus U(-0.05,0.05)
 *         per-voxel noise.  Raw values (not normalised).
 * kind 2: 64 advecting Gaussian blobs (sigma = 0.03*max dim, centres U[0.15,0.85]*dim, 1 voxel/step)
 *         plus 3-octave 4D value noise (spacing 32/2^o voxels, 16/2^o steps, amplitude 0.3*0.5^o);
 *         normalised to [0,1] over the 4D domain.
 * kind 3: flame-like front: 0.5*(1+tanh((xf - x)/4)), xf = 0.08*nx + 2t + 2D value noise of amplitude
 *         0.04*nx (spacing 64 voxels), plus 4-octave value noise (spacing 32/2^o, amplitude 0.05*0.5^o);
 *         normalised to [0,1].
 * kind 4: expanding radial shell exp(-((r - (20 + 2t))/3)^2) around the centre, plus 4-octave value
 *         noise (amplitude 0.1*0.5^o); normalised to [0,1].
 * Blobs contribute inside |x - c|_inf <= ceil(4 sigma) only (part of the definition).
 * Layout out[t][z][y][x], time steps [t0, t1) of a field with nt steps in total.
 */
typedef struct { double cx, cy, cz, dx, dy, dz, sigma, amp; } blob;

static void make_blobs(uint64_t seed, int nb, double sigma, const double lo[3], const double hi[3], blob* b) {
    float u[6];
    for (int i = 0; i < nb; ++i) {
        synth_uniform(seed, 1, (uint64_t)i * 6, 6, 0.0, 1.0, u);
        b[i].cx = lo[0] + (hi[0] - lo[0]) * u[0];
        b[i].cy = lo[1] + (hi[1] - lo[1]) * u[1];
        b[i].cz = lo[2] + (hi[2] - lo[2]) * u[2];
        double z = 2.0 * u[3] - 1.0, phi = 2.0 * M_PI * u[4], r = sqrt(fmax(0.0, 1.0 - z * z));
        b[i].dx = r * cos(phi); b[i].dy = r * sin(phi); b[i].dz = z;
        b[i].sigma = sigma; b[i].amp = 1.0;
    }
}

static void add_blobs(const blob* b, int nb, int64_t nx, int64_t ny, int64_t nz, int64_t t, float* vol) {
    for (int i = 0; i < nb; ++i) {
        double cx = b[i].cx + t * b[i].dx, cy = b[i].cy + t * b[i].dy, cz = b[i].cz + t * b[i].dz;
        int64_t rad = (int64_t)ceil(4.0 * b[i].sigma);
        int64_t x0 = (int64_t)floor(cx) - rad, x1 = (int64_t)floor(cx) + rad + 1;
        int64_t y0 = (int64_t)floor(cy) - rad, y1 = (int64_t)floor(cy) + rad + 1;
        int64_t z0 = (int64_t)floor(cz) - rad, z1 = (int64_t)floor(cz) + rad + 1;
        if (x0 < 0) x0 = 0; if (y0 < 0) y0 = 0; if (z0 < 0) z0 = 0;
        if (x1 > nx - 1) x1 = nx - 1; if (y1 > ny - 1) y1 = ny - 1; if (z1 > nz - 1) z1 = nz - 1;
        double inv = 1.0 / (2.0 * b[i].sigma * b[i].sigma);
#pragma omp parallel for schedule(static)
        for (int64_t z = z0; z <= z1; ++z)
            for (int64_t y = y0; y <= y1; ++y)
                for (int64_t x = x0; x <= x1; ++x) {
                    double d2 = (x - cx) * (x - cx) + (y - cy) * (y - cy) + (z - cz) * (z - cz);
                    vol[(z * ny + y) * nx + x] += (float)(b[i].amp * exp(-d2 * inv));
                }
    }
}

static void add_noise(const noise_lattice* lat, int octaves, double amp0, int64_t nx, int64_t ny, int64_t nz,
                      int64_t t, float* vol) {
    for (int o = 0; o < octaves; ++o) {
        const noise_lattice* L = &lat[o];
        float* sl = lattice_slice(L, t);
        double a = amp0 * pow(0.5, o);
#pragma omp parallel for schedule(static)
        for (int64_t z = 0; z < nz; ++z)
            for (int64_t y = 0; y < ny; ++y)
                for (int64_t x = 0; x < nx; ++x) vol[(z * ny + y) * nx + x] += (float)(a * slice_eval(L, sl, x, y, z));
        free(sl);
    }
}

/* Octave o: spacing sp0/2^o voxels and st0/2^o steps (at least 1), values from stream 10 + o. */
static void make_lattices(uint64_t seed, int octaves, double sp0, double st0, int64_t nx, int64_t ny, int64_t nz,
                          int64_t nt, noise_lattice* lat) {
    for (int o = 0; o < octaves; ++o) {
        double s = sp0 / (double)(1 << o), st = st0 / (double)(1 << o);
        if (st < 1.0) st = 1.0;
        lattice_init(&lat[o], seed, 10 + (uint64_t)o, nx, ny, nz, nt, s, st);
    }
}

int synth_field(int kind, uint64_t seed, int64_t nx, int64_t ny, int64_t nz, int64_t nt, int64_t t0, int64_t t1,
                float* out) {
    if (t0 < 0 || t1 > nt || t0 >= t1 || nx < 2 || ny < 2 || nz < 2) return 1;
    int64_t n3 = nx * ny * nz;
    noise_lattice lat[4];
    const int octaves = kind == 2 ? 3 : (kind == 3 || kind == 4) ? 4 : 0;
    make_lattices(seed, octaves, 32.0, 16.0, nx, ny, nz, nt, lat);
    double mx = (double)(nx > ny ? (nx > nz ? nx : nz) : (ny > nz ? ny : nz));
    for (int64_t t = t0; t < t1; ++t) {
        float* vol = out + (t - t0) * n3;
        memset(vol, 0, (size_t)n3 * sizeof(float));
        if (kind == 1) {
            blob b[4];
            double lo[3] = {8, 8, 8}, hi[3] = {24, 24, 24};
            make_blobs(seed, 4, 3.0, lo, hi, b);
            add_blobs(b, 4, nx, ny, nz, t, vol);
            uint64_t key = stream_key(seed, 3);
#pragma omp parallel for schedule(static)
            for (int64_t i = 0; i < n3; ++i)
                vol[i] += (float)(-0.05 + 0.1 * unit24(rnd64(key, (uint64_t)(t * n3 + i))));
        } else if (kind == 2) {
            blob b[64];
            double lo[3] = {0.15 * nx, 0.15 * ny, 0.15 * nz}, hi[3] = {0.85 * nx, 0.85 * ny, 0.85 * nz};
            make_blobs(seed, 64, 0.03 * mx, lo, hi, b);
            add_blobs(b, 64, nx, ny, nz, t, vol);
            add_noise(lat, 3, 0.3, nx, ny, nz, t, vol);
        } else if (kind == 3) {
            noise_lattice H;   /* 2D height noise over (y, z), reusing a 3D lattice slice at x = 0 */
            lattice_init(&H, seed, 5, 1, ny, nz, 1, 64.0, 1.0);
            float* hs = lattice_slice(&H, 0);
#pragma omp parallel for schedule(static)
            for (int64_t z = 0; z < nz; ++z)
                for (int64_t y = 0; y < ny; ++y) {
                    double xf = 0.08 * nx + 2.0 * t + 0.04 * nx * slice_eval(&H, hs, 0, y, z);
                    for (int64_t x = 0; x < nx; ++x)
                        vol[(z * ny + y) * nx + x] = (float)(0.5 * (1.0 + tanh((xf - x) / 4.0)));
                }
            free(hs); free(H.v);
            add_noise(lat, 4, 0.05, nx, ny, nz, t, vol);
        } else if (kind == 4) {
            double cx = 0.5 * (nx - 1), cy = 0.5 * (ny - 1), cz = 0.5 * (nz - 1), r0 = 20.0 + 2.0 * t;
#pragma omp parallel for schedule(static)
            for (int64_t z = 0; z < nz; ++z)
                for (int64_t y = 0; y < ny; ++y)
                    for (int64_t x = 0; x < nx; ++x) {
                        double r = sqrt((x - cx) * (x - cx) + (y - cy) * (y - cy) + (z - cz) * (z - cz));
                        double q = (r - r0) / 3.0;
                        vol[(z * ny + y) * nx + x] = (float)exp(-q * q);
                    }
            add_noise(lat, 4, 0.1, nx, ny, nz, t, vol);
        } else {
            for (int o = 0; o < octaves; ++o) free(lat[o].v);
            return 2;
        }
    }
    for (int o = 0; o < octaves; ++o) free(lat[o].v);
    return 0;
}

/* Affine rescale in place: v <- (v - lo) / (hi - lo), computed in double, rounded to float. */
void synth_rescale(float* v, int64_t n, double lo, double hi) {
    double inv = 1.0 / (hi - lo);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) v[i] = (float)((v[i] - lo) * inv);
}

void synth_minmax(const float* v, int64_t n, double* lo, double* hi) {
    float a = v[0], b = v[0];
#pragma omp parallel for reduction(min : a) reduction(max : b) schedule(static)
    for (int64_t i = 0; i < n; ++i) { if (v[i] < a) a = v[i]; if (v[i] > b) b = v[i]; }
    *lo = a; *hi = b;
}

static int cmp_f(const void* a, const void* b) {
    float x = *(const float*)a, y = *(const float*)b;
    return (x > y) - (x < y);
}

/* q-quantile of the subsample v[0], v[stride], v[2 stride], ...: element of rank floor(q*(m-1)) after sorting. */
float synth_quantile(const float* v, int64_t n, double q, int64_t stride) {
    int64_t m = (n + stride - 1) / stride;
    float* s = (float*)malloc((size_t)m * sizeof(float));
    for (int64_t i = 0; i < m; ++i) s[i] = v[i * stride];
    qsort(s, (size_t)m, sizeof(float), cmp_f);
    float r = s[(int64_t)floor(q * (double)(m - 1))];
    free(s);
    return r;
}

/* mask[i] = v[i] > thr (u8 0/1); interval form lo < v < hi when hi > lo. */
void synth_mask(const float* v, int64_t n, float thr, float hi, uint8_t* mask) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) mask[i] = (hi > thr) ? (uint8_t)(v[i] > thr && v[i] < hi) : (uint8_t)(v[i] > thr);
}

/*
 * Training targets: the voxel field sampled at FBB-normalised points u in [0,1]^4 (x, y, z, t),
 * trilinear in space and linear in time.  Voxel position p_d = lo_d + u_d * (S_d - 1), time
 * p_t = u_t * (nt - 1); computed in double and rounded to float.  coords: [n][4] float.
 */
void synth_sample(const float* f, int64_t nx, int64_t ny, int64_t nz, int64_t nt, const int64_t lo[3],
                  const int64_t size[3], const float* coords, int64_t n, float* out) {
    const int64_t dims[4] = {nx, ny, nz, nt};
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < n; ++s) {
        int64_t i[4]; double w[4];
        for (int d = 0; d < 4; ++d) {
            double u = coords[s * 4 + d];
            if (!(u > 0.0)) u = 0.0;
            if (u > 1.0) u = 1.0;
            double p = (d < 3) ? lo[d] + u * (double)(size[d] - 1) : u * (double)(nt - 1);
            int64_t c = (int64_t)floor(p);
            if (c > dims[d] - 2) c = dims[d] - 2;
            if (c < 0) c = 0;
            i[d] = c; w[d] = (dims[d] > 1) ? p - (double)c : 0.0;
        }
        double acc = 0.0;
        for (int ct = 0; ct < 2; ++ct)
            for (int cz = 0; cz < 2; ++cz)
                for (int cy = 0; cy < 2; ++cy)
                    for (int cx = 0; cx < 2; ++cx) {
                        int64_t tt = i[3] + ct; if (tt > nt - 1) tt = nt - 1;
                        double wt = (ct ? w[3] : 1 - w[3]) * (cz ? w[2] : 1 - w[2]) * (cy ? w[1] : 1 - w[1]) *
                                    (cx ? w[0] : 1 - w[0]);
                        acc += wt * f[((tt * nz + i[2] + cz) * ny + i[1] + cy) * nx + i[0] + cx];
                    }
        out[s] = (float)acc;
    }
}
