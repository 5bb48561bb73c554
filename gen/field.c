/*
 * Seeded synthetic ensemble fields (input generation only).
 *
 * This file produces the inputs that both the FP64 oracle and the CUDA library
 * consume. It holds none of the correlation method's arithmetic: it only draws
 * noise and shapes it into a smooth random field, the stand-in for the
 * paper's weather ensembles (the real data sets are not available).
 *
 * Recipe (one member m, voxel p = (x, y, z) of a field of size X x Y x Z):
 *   g_m(p)  unit-variance Gaussian random field: white noise convolved with a
 *           separable Gaussian kernel of standard deviation (3, 3, 1) voxels,
 *           truncated at 4 sigma; the kernel is scaled so that the sum of its
 *           squared taps is 1, which gives unit variance.
 *   s_m     one shared latent standard normal per member.
 *   w(x)    ramp 1.5 * x / (X - 1).
 *   f_m(p)  g_m(p) + w(x) * s_m                     for y <  Y/2
 *           g_m(p) + w(x) * (s_m^2 - 1) / sqrt(2)   for y >= Y/2
 * The second half depends on the latent only through its square, so Pearson
 * across the halves is near zero while mutual information is positive.
 *
 * Noise is a counter-based hash of (seed, member, voxel), so any sub-box of the
 * conceptual field can be generated on its own and agrees with the full field.
 * Output layout is [n][bz][by][bx] (member-major, x fastest), fp32.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static uint64_t mix64(uint64_t z) {
    /* SplitMix64 finaliser (Steele, Lea, Flood 2014). */
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double unit_open(uint64_t h) {
    /* (0, 1): 53 random bits, centred in their cell. */
    return ((double)(h >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

static double normal_from_key(uint64_t key) {
    /* Box-Muller on two hashed uniforms. */
    double u1 = unit_open(mix64(key));
    double u2 = unit_open(mix64(key ^ 0xD1B54A32D192ED03ull));
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

static uint64_t voxel_key(uint64_t seed, int64_t m, int64_t gx, int64_t gy, int64_t gz) {
    uint64_t c = ((uint64_t)(gz + 32768) << 42) | ((uint64_t)(gy + 1048576) << 21) |
                 (uint64_t)(gx + 1048576);
    return mix64(mix64(mix64(seed) ^ (uint64_t)m) ^ c);
}

static double latent(uint64_t seed, int64_t m) {
    return normal_from_key(mix64(mix64(seed ^ 0x5851F42D4C957F2Dull) ^ (uint64_t)m));
}

static int kernel_taps(double sigma, double* w) {
    int r = (int)ceil(4.0 * sigma);
    double ss = 0.0;
    for (int d = -r; d <= r; ++d) {
        double v = exp(-(double)(d * d) / (2.0 * sigma * sigma));
        w[d + r] = v;
        ss += v * v;
    }
    double s = 1.0 / sqrt(ss);
    for (int d = 0; d <= 2 * r; ++d) w[d] *= s;
    return r;
}

/*
 * Generate the sub-box [x0, x0+bx) x [y0, y0+by) x [z0, z0+bz) of the field of
 * full size X x Y x Z with n members. out has n*bz*by*bx floats.
 * Returns 0 on success, -1 on bad arguments, -2 on allocation failure.
 */
int gen_field_box(uint64_t seed, int X, int Y, int Z, int n, int x0, int y0, int z0,
                  int bx, int by, int bz, float* out) {
    if (X < 2 || Y < 1 || Z < 1 || n < 1 || bx < 1 || by < 1 || bz < 1) return -1;
    if (x0 < 0 || y0 < 0 || z0 < 0 || x0 + bx > X || y0 + by > Y || z0 + bz > Z) return -1;
    double kx[64], ky[64], kz[64];
    const int rx = kernel_taps(3.0, kx), ry = kernel_taps(3.0, ky), rz = kernel_taps(1.0, kz);
    const int px = bx + 2 * rx, py = by + 2 * ry, pz = bz + 2 * rz;
    int err = 0;
#pragma omp parallel
    {
        double* noise = (double*)malloc(sizeof(double) * (size_t)px * py * pz);
        double* cx = (double*)malloc(sizeof(double) * (size_t)bx * py * pz);
        double* cy = (double*)malloc(sizeof(double) * (size_t)bx * by * pz);
        if (!noise || !cx || !cy) {
#pragma omp atomic write
            err = -2;
        }
#pragma omp for schedule(dynamic, 1)
        for (int m = 0; m < n; ++m) {
            if (err) continue;
            for (int k = 0; k < pz; ++k)
                for (int j = 0; j < py; ++j)
                    for (int i = 0; i < px; ++i)
                        noise[((size_t)k * py + j) * px + i] = normal_from_key(
                            voxel_key(seed, m, x0 - rx + i, y0 - ry + j, z0 - rz + k));
            for (int k = 0; k < pz; ++k)
                for (int j = 0; j < py; ++j)
                    for (int i = 0; i < bx; ++i) {
                        const double* row = noise + ((size_t)k * py + j) * px + i;
                        double acc = 0.0;
                        for (int d = 0; d <= 2 * rx; ++d) acc += kx[d] * row[d];
                        cx[((size_t)k * py + j) * bx + i] = acc;
                    }
            for (int k = 0; k < pz; ++k)
                for (int j = 0; j < by; ++j)
                    for (int i = 0; i < bx; ++i) {
                        double acc = 0.0;
                        for (int d = 0; d <= 2 * ry; ++d)
                            acc += ky[d] * cx[((size_t)k * py + j + d) * bx + i];
                        cy[((size_t)k * by + j) * bx + i] = acc;
                    }
            const double s = latent(seed, m);
            const double s2 = (s * s - 1.0) / sqrt(2.0);
            for (int k = 0; k < bz; ++k)
                for (int j = 0; j < by; ++j)
                    for (int i = 0; i < bx; ++i) {
                        double acc = 0.0;
                        for (int d = 0; d <= 2 * rz; ++d)
                            acc += kz[d] * cy[((size_t)(k + d) * by + j) * bx + i];
                        const int gx = x0 + i, gy = y0 + j;
                        const double w = 1.5 * (double)gx / (double)(X - 1);
                        acc += w * (gy < Y / 2 ? s : s2);
                        out[(((size_t)m * bz + k) * by + j) * bx + i] = (float)acc;
                    }
        }
        free(noise);
        free(cx);
        free(cy);
    }
    return err;
}

/*
 * Cluster fixture in the manner of the paper's Synth1 data set (Section 5.1):
 * at every voxel a blend lambda * d_m + (1 - lambda) * e_m(p) of one shared
 * deterministic sequence d_m and i.i.d. noise e_m(p). lambda is 1 at each of
 * the nc cluster centres (cx, cy, cz, radius) and decays linearly with the
 * l-infinity distance to the nearest centre, reaching 0 at the radius. Voxels
 * with lambda = 1 carry identical member vectors, so their correlation is 1.
 * Output layout [n][Z][Y][X].
 */
int gen_clusters(uint64_t seed, int X, int Y, int Z, int n, const int* centres, int nc,
                 float* out) {
    if (X < 1 || Y < 1 || Z < 1 || n < 2 || nc < 0) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < (int64_t)X * Y * Z; ++p) {
        const int x = (int)(p % X), y = (int)((p / X) % Y), z = (int)(p / ((int64_t)X * Y));
        double lam = 0.0;
        for (int c = 0; c < nc; ++c) {
            int dx = abs(x - centres[4 * c]), dy = abs(y - centres[4 * c + 1]),
                dz = abs(z - centres[4 * c + 2]);
            int d = dx > dy ? dx : dy;
            d = d > dz ? d : dz;
            double l = 1.0 - (double)d / (double)centres[4 * c + 3];
            if (l > lam) lam = l;
        }
        for (int m = 0; m < n; ++m) {
            const double dm = (double)m / (double)(n - 1) * 2.0 - 1.0;
            const double e = normal_from_key(voxel_key(seed, m, x, y, z));
            double v = lam >= 1.0 ? dm : lam * dm + (1.0 - lam) * e;
            out[(size_t)m * X * Y * Z + p] = (float)v;
        }
    }
    return 0;
}
