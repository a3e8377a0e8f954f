// pi_interact.cu -- interaction kernels (arXiv 2406.16091, Sec. 2-5).
//
// For every particle i: n_i = #{j != i : r2_ij < rc2}, S_i = sum K_ij and
// V_i = sum (p_j - p_i) K_ij with K = exp(-r^2/h^2) = 2^(r2 * kscale),
// kscale = -log2(e)/h^2.  The pair test is the frozen FP32 form
// r2 = fma(dz, dz, fma(dy, dy, dx*dx)) < fl32(r_c^2) with d = p_j - p_i in
// FP32, so neighbour counts are exact.  K uses the ex2.approx instruction.
//
// Kernels:
//   k_interact_ppnl   Alg. 1 (Par-Part-NoLoop): one thread per particle,
//                     sources read straight from global memory.  Kept as the
//                     comparator the paper measures its speedups against.
//   k_interact_tiled  reads P, the copy of the sorted particles written by
//                     binning in which every cell is ordered by x and .w
//                     carries the stable slot; every X-row of P is sorted by
//                     x as a whole.  One CTA per X-row of target cells (rows handed out
//                     dynamically), processed in chunks of consecutive cells.
//                     The 9 neighbour rows (y +- 1, z +- 1) of a chunk are
//                     contiguous ranges of P; each is staged into shared memory
//                     with one cp.async.bulk copy (Sec. 5.2 loads pencils along
//                     X; here the whole 3x3 bundle of pencils is loaded at once
//                     because the sorted order makes each one contiguous).
//                     Each thread holds one target in registers and, per
//                     neighbour row, scans only the x-window
//                     [x_i - w_r, x_i + w_r], w_r = sqrt(rc^2 - d_yz^2), where
//                     d_yz is the target's distance to the row in y and z --
//                     sources outside it cannot pass the pair test.
#include "pi_internal.cuh"

namespace pi {

namespace {

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct PlainAcc {
    float v = 0.f;
    __device__ __forceinline__ void add(float t) { v += t; }
    __device__ __forceinline__ void addmul(float a, float b) { v = fmaf(a, b, v); }
    __device__ __forceinline__ float value() const { return v; }
};

// Kahan-compensated FP32 accumulation (precision mode).
struct KahanAcc {
    float v = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float t)
    {
        float y = __fsub_rn(t, c);
        float u = __fadd_rn(v, y);
        c = __fsub_rn(__fsub_rn(u, v), y);
        v = u;
    }
    __device__ __forceinline__ void addmul(float a, float b) { add(__fmul_rn(a, b)); }
    __device__ __forceinline__ float value() const { return v; }
};

template <class Acc>
struct Sums {
    Acc s, vx, vy, vz;
    uint32_t n = 0;

    // One candidate source at FP32 offset (dx, dy, dz) from the target.
    __device__ __forceinline__ void pair(float dx, float dy, float dz, float rc2, float kscale)
    {
        const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
        if (r2 < rc2) {
            const float K = ex2_approx(__fmul_rn(r2, kscale));
            s.add(K);
            vx.addmul(dx, K);
            vy.addmul(dy, K);
            vz.addmul(dz, K);
            n += 1;
        }
    }
};

template <class Acc>
__device__ __forceinline__ void store_out(const InteractArgs& a, uint32_t slot, const Sums<Acc>& r,
                                          float s_bias, uint32_t n_bias)
{
    const uint32_t o = a.original_order ? a.perm[slot] : slot;
    a.S[o] = r.s.value() - s_bias;
    a.Vx[o] = r.vx.value();
    a.Vy[o] = r.vy.value();
    a.Vz[o] = r.vz.value();
    if (a.nbr) a.nbr[o] = r.n - n_bias;
}

// ---- Alg. 1: Par-Part-NoLoop ------------------------------------------------

template <class Acc>
__global__ void __launch_bounds__(128) k_interact_ppnl(InteractArgs a)
{
    if (load_error(a.ctrl)) return;
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.n) return;
    const float xt = a.sx[k], yt = a.sy[k], zt = a.sz[k];
    const int nx = a.g.n[0], ny = a.g.n[1], nz = a.g.n[2];
    const int cx = axis_cell(xt, a.g.lo[0], a.g.inv_w[0], nx);
    const int cy = axis_cell(yt, a.g.lo[1], a.g.inv_w[1], ny);
    const int cz = axis_cell(zt, a.g.lo[2], a.g.inv_w[2], nz);
    Sums<Acc> r;
    for (int bz = max(cz - 1, 0); bz <= min(cz + 1, nz - 1); ++bz)
        for (int by = max(cy - 1, 0); by <= min(cy + 1, ny - 1); ++by) {
            const uint32_t row = (uint32_t)nx * ((uint32_t)by + (uint32_t)ny * (uint32_t)bz);
            const uint32_t j0 = a.offsets[row + max(cx - 1, 0)];
            const uint32_t j1 = a.offsets[row + min(cx + 1, nx - 1) + 1];
            for (uint32_t j = j0; j < j1; ++j) {
                if (j == k) continue;
                r.pair(__fsub_rn(a.sx[j], xt), __fsub_rn(a.sy[j], yt), __fsub_rn(a.sz[j], zt), a.rc2,
                       a.kscale);
            }
        }
    store_out(a, k, r, 0.f, 0u);
}

// ---- tiled interaction ----------------------------------------------------------

constexpr int TT = 128;      // threads per CTA; at most TT targets per chunk
constexpr int CAP = 2048;    // staged particles per chunk (32 KB of float4)
constexpr int MAXLX = 128;   // cells per chunk along X (table size)

struct Tables {
    uint32_t cs[9][MAXLX + 4];  // start of each cell of a row, relative to the row
    uint32_t gbeg[9];           // first index of each row in P
    int sbeg[9];                // first index of each row in the staged buffer
    int rlen[9];                // particles in each row (0 for rows outside the grid)
    int xa, xb;                 // source cells [xa, xb] of every row
    int x1;                     // end of the target cells of the chunk
    int mode;                   // 0: staged in shared memory, 1: read from global
    int total;                  // staged particles
    uint32_t row;               // current X-row
    int failed;                 // a bounded wait ran out: the CTA stops
};

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void bar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void bar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool bar_try_wait(uint64_t* bar, uint32_t phase)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    return done != 0;
}

// Waits for the staged copies of this chunk; false if the wait ran out.
__device__ __forceinline__ bool bar_wait_bounded(uint64_t* bar, uint32_t phase, uint64_t limit_ns)
{
    if (bar_try_wait(bar, phase)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (bar_try_wait(bar, phase)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// Picks the chunk [x0, x1) of target cells (warp 0).  Largest x1 such that
// the chunk has at most TT targets and its 9 source rows hold at most CAP
// particles; a single cell whose rows exceed CAP is read from global memory.
__device__ void choose_chunk(const InteractArgs& a, Tables& t, int x0, int cy, int cz, unsigned lane)
{
    const int nx = a.g.n[0], ny = a.g.n[1], nz = a.g.n[2];
    const uint32_t rb0 = (uint32_t)nx * ((uint32_t)cy + (uint32_t)ny * (uint32_t)cz);
    const uint32_t tgt0 = a.offsets[rb0 + x0];
    const int xmax = min(nx, x0 + MAXLX);
    int best = 0;            // largest valid x1 found
    bool first_fits = true;  // rows of [x0, x0+1) fit in CAP
    for (int base = x0 + 1; base <= xmax; base += 32) {
        const int x1 = base + (int)lane;
        bool valid = false;
        bool fits = true;
        if (x1 <= xmax) {
            const uint32_t targets = a.offsets[rb0 + x1] - tgt0;
            uint32_t staged = 0;
            const int xa = max(x0 - 1, 0), xb = min(x1, nx - 1);
#pragma unroll
            for (int r = 0; r < 9; ++r) {
                const int by = cy + r % 3 - 1, bz = cz + r / 3 - 1;
                if (by < 0 || by >= ny || bz < 0 || bz >= nz) continue;
                const uint32_t rb = (uint32_t)nx * ((uint32_t)by + (uint32_t)ny * (uint32_t)bz);
                staged += a.offsets[rb + xb + 1] - a.offsets[rb + xa];
            }
            fits = staged <= (uint32_t)CAP;
            valid = fits && targets <= (uint32_t)TT;
        }
        const unsigned vm = __ballot_sync(0xffffffffu, valid);
        if (base == x0 + 1) first_fits = __shfl_sync(0xffffffffu, fits, 0);
        if (vm) best = base + 31 - __clz(vm);
        if (vm != 0xffffffffu) break;
    }
    if (lane == 0) {
        if (best == 0) {
            t.x1 = x0 + 1;
            t.mode = first_fits ? 0 : 1;
        } else {
            t.x1 = best;
            t.mode = 0;
        }
    }
}

// Sums of one target over the 9 rows.  SRC is the staged buffer (smem) or P.
template <class Acc, bool SMEM>
__device__ __forceinline__ void target_sums(const InteractArgs& a, const Tables& t, const float4* src,
                                            float4 me, int cy, int cz, Sums<Acc>& r)
{
    const float xt = me.x, yt = me.y, zt = me.z;
    const float wy = 1.0f / a.g.inv_w[1], wz = 1.0f / a.g.inv_w[2];
    // distances to the lower / upper faces of the own cell in y and z
    const float fy_lo = fmaxf(yt - fmaf((float)cy, wy, a.g.lo[1]) - a.slack, 0.f);
    const float fy_hi = fmaxf(fmaf((float)(cy + 1), wy, a.g.lo[1]) - yt - a.slack, 0.f);
    const float fz_lo = fmaxf(zt - fmaf((float)cz, wz, a.g.lo[2]) - a.slack, 0.f);
    const float fz_hi = fmaxf(fmaf((float)(cz + 1), wz, a.g.lo[2]) - zt - a.slack, 0.f);
    const float rcm2 = a.rc2 * 1.00002f;
#pragma unroll 1
    for (int rr = 0; rr < 9; ++rr) {
        const int len = t.rlen[rr];
        if (len == 0) continue;
        const int dy = rr % 3 - 1, dz = rr / 3 - 1;
        const float ey = dy < 0 ? fy_lo : (dy > 0 ? fy_hi : 0.f);
        const float ez = dz < 0 ? fz_lo : (dz > 0 ? fz_hi : 0.f);
        const float d2 = fmaf(ey, ey, ez * ez);
        if (d2 >= rcm2) continue;
        const float w = __fsqrt_rn(rcm2 - d2) + a.slack;
        const float xlo = xt - w, xhi = xt + w;
        // first source with x >= xlo: start in the cell of xlo (cells are
        // monotone in x), then binary search inside that cell
        int k = axis_cell(xlo, a.g.lo[0], a.g.inv_w[0], a.g.n[0]) - t.xa;
        k = max(k, 0);
        const int kmax = t.xb - t.xa;
        k = min(k, kmax);
        const float4* rowg = SMEM ? (src + t.sbeg[rr]) : (src + t.gbeg[rr]);
        int lo = t.cs[rr][k], hi = t.cs[rr][k + 1];
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (rowg[mid].x < xlo) lo = mid + 1;
            else hi = mid;
        }
        for (int j = lo; j < len; ++j) {
            const float4 s = rowg[j];
            if (s.x > xhi) break;
            r.pair(__fsub_rn(s.x, xt), __fsub_rn(s.y, yt), __fsub_rn(s.z, zt), a.rc2, a.kscale);
        }
    }
}

template <class Acc>
__global__ void __launch_bounds__(TT) k_interact_tiled(InteractArgs a)
{
    __shared__ __align__(16) float4 buf[CAP];
    __shared__ Tables t;
    __shared__ __align__(8) uint64_t bar;

    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctrl->work[(a.seq + 1u) & 1u] = 0u;
    if (load_error(a.ctrl)) return;
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const int nx = a.g.n[0], ny = a.g.n[1], nz = a.g.n[2];
    const uint32_t rows = (uint32_t)ny * (uint32_t)nz;
    // K(0) of this hardware path: the self pair adds exactly this to S
    const float k0 = ex2_approx(0.f);

    if (threadIdx.x == 0) {
        t.failed = 0;
        bar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t phase = 0;

    for (;;) {
        if (threadIdx.x == 0) t.row = atomicAdd(&a.ctrl->work[a.seq & 1u], 1u);
        __syncthreads();
        const uint32_t row = t.row;
        if (row >= rows || t.failed) break;
        const int cy = (int)(row % (uint32_t)ny), cz = (int)(row / (uint32_t)ny);
        const uint32_t rb0 = (uint32_t)nx * row;

        for (int x0 = 0; x0 < nx;) {
            if (warp == 0) choose_chunk(a, t, x0, cy, cz, lane);
            __syncthreads();
            const int x1 = t.x1;
            const int xa = max(x0 - 1, 0), xb = min(x1, nx - 1);
            // row ranges (warp 0, one lane per row)
            if (warp == 0) {
                uint32_t gb = 0, len = 0;
                if (lane < 9) {
                    const int by = cy + (int)lane % 3 - 1, bz = cz + (int)lane / 3 - 1;
                    if (by >= 0 && by < ny && bz >= 0 && bz < nz) {
                        const uint32_t rb = (uint32_t)nx * ((uint32_t)by + (uint32_t)ny * (uint32_t)bz);
                        gb = a.offsets[rb + xa];
                        len = a.offsets[rb + xb + 1] - gb;
                    }
                }
                uint32_t incl = len;
#pragma unroll
                for (int o = 1; o < 16; o <<= 1) {
                    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= (unsigned)o) incl += v;
                }
                if (lane < 9) {
                    t.gbeg[lane] = gb;
                    t.rlen[lane] = (int)len;
                    t.sbeg[lane] = (int)(incl - len);
                }
                if (lane == 8) t.total = (int)incl;
                if (lane == 0) {
                    t.xa = xa;
                    t.xb = xb;
                }
            }
            __syncthreads();
            // per-row cell start tables (relative to the row start)
            const int ncell = xb - xa + 1;
            for (int e = threadIdx.x; e < 9 * (ncell + 1); e += TT) {
                const int rr = e / (ncell + 1), k = e % (ncell + 1);
                const int by = cy + rr % 3 - 1, bz = cz + rr / 3 - 1;
                uint32_t v = 0;
                if (by >= 0 && by < ny && bz >= 0 && bz < nz) {
                    const uint32_t rb = (uint32_t)nx * ((uint32_t)by + (uint32_t)ny * (uint32_t)bz);
                    v = a.offsets[rb + xa + k] - t.gbeg[rr];
                }
                t.cs[rr][k] = v;
            }
            const int mode = t.mode;
            if (mode == 0 && threadIdx.x == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                bar_expect_tx(&bar, (uint32_t)t.total * 16u);
                for (int rr = 0; rr < 9; ++rr)
                    if (t.rlen[rr] > 0)
                        bulk_g2s(&buf[t.sbeg[rr]], a.P + t.gbeg[rr], (uint32_t)t.rlen[rr] * 16u, &bar);
            }
            __syncthreads();
            if (mode == 0) {
                if (!bar_wait_bounded(&bar, phase, a.wait_limit_ns)) {
                    t.failed = 1;
                    atomicOr(&a.ctrl->error, ERR_TIMEOUT);
                    // let the copies in flight land before the CTA exits
                    bar_wait_bounded(&bar, phase, a.wait_limit_ns);
                }
                phase ^= 1u;
            }
            __syncthreads();  // t.failed is uniform from here on
            // targets: cells [x0, x1) of the centre row (row 4)
            const uint32_t tb = a.offsets[rb0 + x0], te = a.offsets[rb0 + x1];
            const int tloc = (int)(tb - t.gbeg[4]);
            const int ntarget = (int)(te - tb);
            if (!t.failed) {
                for (int q = threadIdx.x; q < ntarget; q += TT) {
                    Sums<Acc> r;
                    float4 me;
                    if (mode == 0) {
                        me = buf[t.sbeg[4] + tloc + q];
                        target_sums<Acc, true>(a, t, buf, me, cy, cz, r);
                    } else {
                        me = a.P[tb + q];
                        target_sums<Acc, false>(a, t, a.P, me, cy, cz, r);
                    }
                    store_out(a, __float_as_uint(me.w), r, k0, 1u);
                }
            }
            __syncthreads();
            x0 = x1;
        }
    }
}

}  // namespace

cudaError_t launch_interact_ppnl(const InteractArgs& a, bool kahan, int num_sms, cudaStream_t s,
                                 int* launches)
{
    (void)num_sms;
    const unsigned blocks = (unsigned)((a.n + 127) / 128);
    if (kahan) k_interact_ppnl<KahanAcc><<<blocks, 128, 0, s>>>(a);
    else k_interact_ppnl<PlainAcc><<<blocks, 128, 0, s>>>(a);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_interact_tiled(const InteractArgs& a, bool kahan, int num_sms, cudaStream_t s,
                                  int* launches)
{
    const uint32_t rows = (uint32_t)a.g.n[1] * (uint32_t)a.g.n[2];
    int per_sm = 0;
    if (kahan)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_interact_tiled<KahanAcc>, TT, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_interact_tiled<PlainAcc>, TT, 0);
    if (per_sm < 1) per_sm = 1;
    uint64_t grid = (uint64_t)num_sms * per_sm;
    if (grid > rows) grid = rows;
    if (grid < 1) grid = 1;
    if (kahan) k_interact_tiled<KahanAcc><<<(unsigned)grid, TT, 0, s>>>(a);
    else k_interact_tiled<PlainAcc><<<(unsigned)grid, TT, 0, s>>>(a);
    *launches += 1;
    return cudaGetLastError();
}

}  // namespace pi
