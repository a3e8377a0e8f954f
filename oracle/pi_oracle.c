/*
 * pi_oracle.c -- plain, slow, FP64 CPU oracle for cutoff-radius pair
 * interactions on a regular cell grid (arXiv 2406.16091).
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load or call this file.  It
 * shares no code, header, helper or constant with the CUDA library, and the
 * CUDA library never calls it.
 *
 * What it computes follows the paper's statement of the problem:
 *   Sec. 2 (Background): for N particles, every pair (i, j) with i != j and
 *     r_ij < r_c interacts through a kernel K(r_ij); positions live in SoA
 *     arrays; each particle gets a cell index from its position, cells are
 *     counted, the counts are prefix-summed (Fig. 1: the offset array has C+1
 *     entries, the last one is N) and particles are moved into cell order in
 *     a secondary array; then every particle interacts with the particles of
 *     its own cell and of the neighbouring cells.
 *   Sec. 3 (Problem statement): the cell width is at least r_c, so all the
 *     partners of a particle lie in its own cell or the 26 adjacent ones;
 *     outputs are per-particle physical values in SoA form.
 *   Alg. 5, Sec. 5.2: neighbour cells are clipped at the box faces
 *     (Max(0, .) / Min(limit, .)), i.e. the box is not periodic.
 *
 * Readings where the paper is silent:
 *   - K is the Gaussian exp(-r^2/h^2) by default; outputs S_i = sum K and
 *     V_i = sum (p_j - p_i) K (the paper's Lennard-Jones constants are not
 *     fixed by its text).  The other kernels, for the comparisons of
 *     Sec. 7.1-7.2: Lennard-Jones 4 E0 ((sigma/r)^12 - (sigma/r)^6) with
 *     E0 = 1, sigma = h and r^2 softened to r^2 + sigma^2/100 (Sec. 7.1 says
 *     a softening is used without giving it); the low-FLOP kernel K = 1;
 *     the high-FLOP kernel, whose value is the Lennard-Jones one (its extra
 *     work changes nothing in the result).
 *   - Grid: n_d = max(1, floor((hi_d - lo_d) / r_c)) in FP64, so the cell
 *     width is >= r_c.
 *   - Cell index, in FP32: c_d = clamp(floor((x_d - lo_d) * inv_w_d), 0,
 *     n_d - 1), inv_w_d = fl32(n_d / (hi_d - lo_d)), cell = cx + nx*(cy + ny*cz)
 *     (X fastest, so an X-row of cells is contiguous after sorting, Sec. 5.1).
 *   - Cutoff predicate, frozen in FP32 so that neighbour counts are exact on
 *     both sides: d = x_j - x_i per axis (FP32), r2 = fma(dz,dz,fma(dy,dy,dx*dx)),
 *     pair iff r2 < fl32(r_c * r_c).
 *   - Within a cell, particles keep their input order (stable scatter).
 *   - Self-exclusion is by index: distinct coincident particles interact.
 *
 * Everything is sequential except the optional OpenMP loop over target cells
 * in pio_interact (each target is still summed in one fixed order, so the
 * result does not depend on the thread count).  Build with
 * -ffp-contract=off so the FP32 steps are not fused behind our back.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PIO_OK 0
#define PIO_BAD_ARG 1
#define PIO_OUT_OF_BOX 3

/* Number of threads an OpenMP loop will use (1 without OpenMP). */
int pio_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void pio_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Grid dimensions: cell width >= r_c along every axis (Sec. 3). */
int pio_grid_dims(const float lo[3], const float hi[3], float rc, int32_t dims[3])
{
    if (!(rc > 0.0f) || isinf(rc)) return PIO_BAD_ARG;
    for (int d = 0; d < 3; ++d) {
        double len = (double)hi[d] - (double)lo[d];
        if (!(len > 0.0) || isinf(len)) return PIO_BAD_ARG;
        double n = floor(len / (double)rc);
        if (n < 1.0) n = 1.0;
        if (n > 2147483647.0) return PIO_BAD_ARG;
        dims[d] = (int32_t)n;
    }
    return PIO_OK;
}

/* Cell of one position, Sec. 2 ("compute its cell index using its physical
 * position, without moving the particles"), with the FP32 reading above.
 * Returns -1 when the position is outside [lo, hi) on some axis (or NaN). */
static int64_t cell_of(float x, float y, float z, const float lo[3], const float hi[3],
                       const int32_t dims[3])
{
    float p[3] = {x, y, z};
    int64_t c[3];
    for (int d = 0; d < 3; ++d) {
        if (!(p[d] >= lo[d] && p[d] < hi[d])) return -1;
        float inv_w = (float)((double)dims[d] / ((double)hi[d] - (double)lo[d]));
        float rel = p[d] - lo[d];        /* FP32, round to nearest */
        float scaled = rel * inv_w;      /* FP32, round to nearest */
        int64_t k = (int64_t)floorf(scaled);
        if (k < 0) k = 0;
        if (k > dims[d] - 1) k = dims[d] - 1;
        c[d] = k;
    }
    return c[0] + (int64_t)dims[0] * (c[1] + (int64_t)dims[1] * c[2]);
}

/* Cell index of every particle.  Returns PIO_OUT_OF_BOX (and writes cell 0
 * for that particle) if any position is outside the box. */
int pio_cell_index(const float* x, const float* y, const float* z, int64_t n,
                   const float lo[3], const float hi[3], const int32_t dims[3],
                   uint32_t* cell)
{
    int status = PIO_OK;
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = cell_of(x[i], y[i], z[i], lo, hi, dims);
        if (c < 0) { status = PIO_OUT_OF_BOX; c = 0; }
        cell[i] = (uint32_t)c;
    }
    return status;
}

/* Exclusive prefix sum with C+1 outputs, offsets[C] = total (Fig. 1).
 * Plain sequential loop: the definition written out. */
void pio_exclusive_scan(const uint32_t* counts, int64_t C, uint32_t* offsets)
{
    uint64_t run = 0;
    for (int64_t c = 0; c < C; ++c) {
        offsets[c] = (uint32_t)run;
        run += counts[c];
    }
    offsets[C] = (uint32_t)run;
}

/* Binning (Sec. 2): cell index, per-cell count, exclusive scan, then a
 * scatter into cell order.  The scatter walks the particles in input order
 * and hands out slots with a per-cell cursor, so the order inside a cell is
 * the input order (stable counting sort).  Also returns M_C, the largest cell
 * count (Sec. 5.1 keeps it while scanning).  Outputs:
 *   counts[C], offsets[C+1], perm[n] (sorted slot -> input index),
 *   sx/sy/sz[n] (positions in sorted order), *max_per_cell. */
int pio_bin(const float* x, const float* y, const float* z, int64_t n,
            const float lo[3], const float hi[3], const int32_t dims[3],
            uint32_t* counts, uint32_t* offsets, uint32_t* perm,
            float* sx, float* sy, float* sz, uint32_t* max_per_cell)
{
    int64_t C = (int64_t)dims[0] * dims[1] * dims[2];
    uint32_t* cell = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    uint32_t* cursor = (uint32_t*)calloc((size_t)C, sizeof(uint32_t));
    if (!cell || !cursor) { free(cell); free(cursor); return PIO_BAD_ARG; }

    int status = pio_cell_index(x, y, z, n, lo, hi, dims, cell);

    memset(counts, 0, sizeof(uint32_t) * (size_t)C);
    for (int64_t i = 0; i < n; ++i) counts[cell[i]] += 1;

    pio_exclusive_scan(counts, C, offsets);

    uint32_t m = 0;
    for (int64_t c = 0; c < C; ++c) if (counts[c] > m) m = counts[c];
    *max_per_cell = m;

    for (int64_t i = 0; i < n; ++i) {
        uint32_t c = cell[i];
        uint32_t slot = offsets[c] + cursor[c];
        cursor[c] += 1;
        perm[slot] = (uint32_t)i;
        sx[slot] = x[i];
        sy[slot] = y[i];
        sz[slot] = z[i];
    }
    free(cell);
    free(cursor);
    return status;
}

/* The frozen FP32 cutoff predicate (reading above).  dx, dy, dz are the FP32
 * differences x_j - x_i. */
static int within_cutoff(float dx, float dy, float dz, float rc2)
{
    float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    return r2 < rc2;
}

#define PIO_GAUSSIAN 0
#define PIO_LJ 1
#define PIO_LOWFLOP 2
#define PIO_HIGHFLOP 3

/* K for a pair at squared distance r2 (FP64).  *mag is the size the error of
 * an FP32 evaluation scales with: |K| for the Gaussian and the constant, and
 * for Lennard-Jones the sum of the magnitudes of its two terms, 4 (s^6 + s^3),
 * because 4 (s^6 - s^3) cancels near its zero crossing. */
static double kernel_value(int kernel, double r2, double h, double* mag)
{
    if (kernel == PIO_LJ || kernel == PIO_HIGHFLOP) {
        double sig2 = h * h;
        double s = sig2 / (r2 + sig2 / 100.0);
        double s3 = s * s * s;
        double s6 = s3 * s3;
        *mag = 4.0 * (s6 + s3);
        return 4.0 * (s6 - s3);
    }
    if (kernel == PIO_LOWFLOP) {
        *mag = 1.0;
        return 1.0;
    }
    {
        double K = exp(-r2 / (h * h));
        *mag = K;
        return K;
    }
}

/* For every particle k in sorted order: neighbour count, S = sum K,
 * V = sum (p_j - p_k) K over j != k in the clipped 27-cell stencil with the
 * FP32 predicate, all sums in FP64 (exact differences of the FP32 positions).
 * Also returns the sums of |term| per output (the normaliser of the
 * tolerance) and the number of candidate pairs looked at (j != k in the
 * stencil).  Any of the optional outputs may be NULL. */
int pio_interact(const float* sx, const float* sy, const float* sz, int64_t n,
                 const uint32_t* offsets, const int32_t dims[3], float rc, float h, int kernel,
                 double* S, double* Vx, double* Vy, double* Vz, uint32_t* nbr,
                 double* absS, double* absVx, double* absVy, double* absVz,
                 uint64_t* candidates)
{
    if (!(rc > 0.0f) || !(h > 0.0f)) return PIO_BAD_ARG;
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    const int64_t C = nx * ny * nz;
    if ((int64_t)offsets[C] != n) return PIO_BAD_ARG;
    const float rc2 = rc * rc;  /* FP32 product, round to nearest */
    uint64_t total_candidates = 0;

#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total_candidates)
#endif
    for (int64_t c = 0; c < C; ++c) {
        int64_t cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
        for (int64_t k = offsets[c]; k < (int64_t)offsets[c + 1]; ++k) {
            const float xk = sx[k], yk = sy[k], zk = sz[k];
            double s = 0.0, vx = 0.0, vy = 0.0, vz = 0.0;
            double as = 0.0, avx = 0.0, avy = 0.0, avz = 0.0;
            uint32_t cnt = 0;
            for (int64_t bz = cz - 1; bz <= cz + 1; ++bz) {
                if (bz < 0 || bz >= nz) continue;
                for (int64_t by = cy - 1; by <= cy + 1; ++by) {
                    if (by < 0 || by >= ny) continue;
                    for (int64_t bx = cx - 1; bx <= cx + 1; ++bx) {
                        if (bx < 0 || bx >= nx) continue;
                        int64_t b = bx + nx * (by + ny * bz);
                        for (int64_t j = offsets[b]; j < (int64_t)offsets[b + 1]; ++j) {
                            if (j == k) continue;
                            total_candidates += 1;
                            float dx = sx[j] - xk, dy = sy[j] - yk, dz = sz[j] - zk;
                            if (!within_cutoff(dx, dy, dz, rc2)) continue;
                            double ddx = (double)sx[j] - (double)xk;
                            double ddy = (double)sy[j] - (double)yk;
                            double ddz = (double)sz[j] - (double)zk;
                            double r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                            double mag;
                            double K = kernel_value(kernel, r2, (double)h, &mag);
                            cnt += 1;
                            s += K;
                            vx += ddx * K;
                            vy += ddy * K;
                            vz += ddz * K;
                            as += mag;
                            avx += fabs(ddx) * mag;
                            avy += fabs(ddy) * mag;
                            avz += fabs(ddz) * mag;
                        }
                    }
                }
            }
            if (S) S[k] = s;
            if (Vx) Vx[k] = vx;
            if (Vy) Vy[k] = vy;
            if (Vz) Vz[k] = vz;
            if (nbr) nbr[k] = cnt;
            if (absS) absS[k] = as;
            if (absVx) absVx[k] = avx;
            if (absVy) absVy[k] = avy;
            if (absVz) absVz[k] = avz;
        }
    }
    if (candidates) *candidates = total_candidates;
    return PIO_OK;
}

/* O(N^2) brute force over the input order with the same FP32 predicate and
 * FP64 sums: the problem definition of Sec. 2 with no grid at all. */
int pio_brute(const float* x, const float* y, const float* z, int64_t n, float rc, float h,
              int kernel, double* S, double* Vx, double* Vy, double* Vz, uint32_t* nbr)
{
    if (!(rc > 0.0f) || !(h > 0.0f)) return PIO_BAD_ARG;
    const float rc2 = rc * rc;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0, vx = 0.0, vy = 0.0, vz = 0.0;
        uint32_t cnt = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            float dx = x[j] - x[i], dy = y[j] - y[i], dz = z[j] - z[i];
            if (!within_cutoff(dx, dy, dz, rc2)) continue;
            double ddx = (double)x[j] - (double)x[i];
            double ddy = (double)y[j] - (double)y[i];
            double ddz = (double)z[j] - (double)z[i];
            double mag;
            double K = kernel_value(kernel, ddx * ddx + ddy * ddy + ddz * ddz, (double)h, &mag);
            cnt += 1;
            s += K;
            vx += ddx * K;
            vy += ddy * K;
            vz += ddz * K;
        }
        S[i] = s;
        Vx[i] = vx;
        Vy[i] = vy;
        Vz[i] = vz;
        nbr[i] = cnt;
    }
    return PIO_OK;
}
