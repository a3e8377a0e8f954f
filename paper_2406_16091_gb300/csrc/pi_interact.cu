// pi_interact.cu -- interaction kernels (arXiv 2406.16091, Sec. 2-5).
//
// For every particle i: n_i = #{j != i : r2_ij < rc2}, S_i = sum K_ij and
// V_i = sum (p_j - p_i) K_ij.  The pair test is the frozen FP32 form
// r2 = fma(dz, dz, fma(dy, dy, dx*dx)) < fl32(r_c^2) with d = p_j - p_i in
// FP32, so neighbour counts are exact.  K is one of
//   Gaussian       exp(-r^2/h^2) = 2^(r2 t), t = -log2(e)/h^2 (ex2.approx)
//   Lennard-Jones  4 (s^6 - s^3), s = sigma^2 / (r^2 + sigma^2/100),
//                  sigma = h (the Sec. 7.1 potential with E0 = 1 and a
//                  softening of sigma/10)
//   low-FLOP       1 (Sec. 7.2's cheap synthetic kernel: S counts, V sums
//                  the offsets)
//   high-FLOP      Lennard-Jones followed by 75 fused multiply-adds by an
//                  opaque 1 and 0 (Sec. 7.2's expensive synthetic kernel:
//                  the value is unchanged, the work is 150 FLOP more)
// Every kernel works on several independent systems at once: particle,
// cell and X-row indices are global over the concatenated systems.
//
// Kernels:
//   k_interact_ppnl   Alg. 1 (Par-Part-NoLoop): one thread per particle,
//                     sources read straight from global memory.  Kept as the
//                     comparator the paper measures its speedups against.
//   k_interact_tiled  reads P, the x-ordered copy written by binning: the
//                     sorted particles with every cell ordered by x, as float4
//                     (x, y, z, stable slot); every X-row of P is sorted by x
//                     as a whole.  Work items are segments of an X-row of
//                     target cells, handed out dynamically from one queue
//                     over all systems, and processed in chunks of
//                     consecutive cells.  The 9 neighbour rows (y +- 1,
//                     z +- 1) of a chunk are contiguous ranges of P, each
//                     staged into shared memory with one cp.async.bulk copy
//                     (Sec. 5.2 loads pencils along X; here
//                     the whole 3x3 bundle of pencils is loaded at once
//                     because the sorted order makes each one contiguous).
//                     Each thread holds one target in registers and, per
//                     neighbour row, scans only the x-window
//                     [x_i - w_r, x_i + w_r], w_r = sqrt(rc^2 - d_yz^2), where
//                     d_yz is the target's distance to the row in y and z:
//                     sources outside it cannot pass the pair test.  Pairs
//                     of candidates are evaluated with packed f32x2
//                     arithmetic.
#include <type_traits>

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

// Value of the interaction kernel for one pair inside the cutoff; t is the
// system's scale (Gaussian: -log2(e)/h^2; Lennard-Jones: sigma^2).
template <int KERNEL>
__device__ __forceinline__ float kernel_value(float r2, float t, float one, float zero)
{
    if constexpr (KERNEL == KERNEL_GAUSSIAN) {
        return ex2_approx(__fmul_rn(r2, t));
    } else if constexpr (KERNEL == KERNEL_LOWFLOP) {
        return 1.0f;
    } else {
        const float rs2 = __fmaf_rn(0.01f, t, r2);
        const float sr = __fmul_rn(t, __frcp_rn(rs2));
        const float s3 = __fmul_rn(__fmul_rn(sr, sr), sr);
        float K = __fmul_rn(4.0f, __fsub_rn(__fmul_rn(s3, s3), s3));
        if constexpr (KERNEL == KERNEL_HIGHFLOP) {
#pragma unroll
            for (int i = 0; i < 75; ++i) K = __fmaf_rn(K, one, zero);
        }
        return K;
    }
}

// Scale of the kernel and the opaque constants of the high-FLOP kernel.
struct KParams {
    float t, one, zero;
};

// Where the tiled kernel excludes the self pair by identity instead of
// adding K(0) and taking it off again: kernels whose value at r = 0 is far
// larger than their typical sum (Lennard-Jones), and the compensated
// precision mode, where taking K(0) off would cost the accuracy of particles
// whose sum is small next to K(0).
template <int KERNEL, class Acc>
__host__ __device__ constexpr bool self_by_identity()
{
    return KERNEL == KERNEL_LJ || KERNEL == KERNEL_HIGHFLOP || std::is_same<Acc, KahanAcc>::value;
}

// Per-target accumulators of one interaction kernel.
template <class Acc, int KERNEL>
struct Sums {
    Acc s, vx, vy, vz;
    uint32_t n = 0;

    __device__ __forceinline__ void add(float dx, float dy, float dz, float K, bool in)
    {
        s.add(K);
        vx.addmul(dx, K);
        vy.addmul(dy, K);
        vz.addmul(dz, K);
        n += in ? 1u : 0u;
    }

    // One candidate without a branch: K is computed for every candidate and
    // zeroed when the pair test fails (the tiled kernel's inner loop, where
    // a divergent branch per candidate costs more than the kernel value).
    __device__ __forceinline__ void pair_nb(float dx, float dy, float dz, float rc2, const KParams& kp,
                                            bool self = false)
    {
        const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
        const bool in = (r2 < rc2) && !self;
        const float e = kernel_value<KERNEL>(r2, kp.t, kp.one, kp.zero);
        add(dx, dy, dz, in ? e : 0.f, in);
    }

    // One candidate source at FP32 offset (dx, dy, dz) from the target.
    __device__ __forceinline__ void pair(float dx, float dy, float dz, float rc2, const KParams& kp)
    {
        const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
        if (r2 < rc2) add(dx, dy, dz, kernel_value<KERNEL>(r2, kp.t, kp.one, kp.zero), true);
    }
};

template <class Acc, int KERNEL>
__device__ __forceinline__ void store_out(const InteractArgs& a, uint32_t slot,
                                          const Sums<Acc, KERNEL>& r, float s_bias, uint32_t n_bias)
{
    const uint32_t o = a.original_order ? a.perm[slot] : slot;
    a.S[o] = r.s.value() - s_bias;
    a.Vx[o] = r.vx.value();
    a.Vy[o] = r.vy.value();
    a.Vz[o] = r.vz.value();
    if (a.nbr) a.nbr[o] = r.n - n_bias;
}

// ---- Alg. 1: Par-Part-NoLoop ------------------------------------------------

template <class Acc, int KERNEL>
__global__ void __launch_bounds__(128) k_interact_ppnl(InteractArgs a)
{
    if (load_error(a.ctrl)) return;
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.n) return;
    const int sid = a.sy.S == 1 ? 0 : find_system(a.sy.pbase, a.sy.S, k);
    const SysDesc& d = a.sy.sys[sid];
    const Grid& g = d.g;
    const float xt = a.sx[k], yt = a.sy_pos[k], zt = a.sz[k];
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int cx = axis_cell(xt, g.lo[0], g.inv_w[0], nx);
    const int cy = axis_cell(yt, g.lo[1], g.inv_w[1], ny);
    const int cz = axis_cell(zt, g.lo[2], g.inv_w[2], nz);
    Sums<Acc, KERNEL> r;
    const KParams kp{a.kscale ? a.kscale[sid] : a.kscale0, a.one, a.zero};
    for (int bz = max(cz - 1, 0); bz <= min(cz + 1, nz - 1); ++bz)
        for (int by = max(cy - 1, 0); by <= min(cy + 1, ny - 1); ++by) {
            const uint32_t row = d.cell_base + (uint32_t)nx * ((uint32_t)by + (uint32_t)ny * (uint32_t)bz);
            const uint32_t j0 = a.offsets[row + max(cx - 1, 0)];
            const uint32_t j1 = a.offsets[row + min(cx + 1, nx - 1) + 1];
            for (uint32_t j = j0; j < j1; ++j) {
                if (j == k) continue;
                r.pair(__fsub_rn(a.sx[j], xt), __fsub_rn(a.sy_pos[j], yt), __fsub_rn(a.sz[j], zt), d.rc2, kp);
            }
        }
    store_out(a, k, r, 0.f, 0u);
}

// ---- tiled interaction ----------------------------------------------------------

// Tile shapes: threads per CTA (= targets per chunk) and staged particles per
// chunk.  The autotuner (pi_autotune) picks one per context; every shape
// gives the same per-target summation order, so the results are identical.
template <int TT_, int CAP_, int MINB_>
struct Tile {
    static constexpr int TT = TT_;
    static constexpr int CAP = CAP_;
    static constexpr int MINB = MINB_;  // CTAs per SM the register budget is sized for
};
using Tile64 = Tile<64, 640, 16>;
using Tile128 = Tile<128, 1280, 8>;
using Tile256 = Tile<256, 2560, 4>;

constexpr int MAXLX = 64;                   // target cells per chunk along X
constexpr int BPC = 4;                      // x-bins per cell in the staged-row lookup
constexpr int RBINS = (MAXLX + 2) * BPC + 2;

// One chunk: target cells [x0, x1) of an X-row, source cells [xa, xb] of the
// 9 neighbour rows (row r has dy = r % 3 - 1, dz = r / 3 - 1).  Row r holds
// the particles [gbeg, gbeg + rlen) of P and lands at sbeg in the staging
// buffer (float4 entries are 16 bytes, so every copy is 16-byte aligned).
struct Plan {
    uint32_t gbeg[9];
    int rlen[9];
    int sbeg[9];
    int xa, xb;
    int x1;
    int mode;   // 0: rows staged in shared memory, 1: rows read from global
    int total;  // staged particles
};

template <int CAP>
struct Smem {
    float4 buf[CAP + 1];  // staged rows; one spare slot keeps a read one past the end inside
    union {
        // mode 0: per row, first staged index (absolute) whose x-bin is >= b
        uint16_t bin[9][RBINS];
        // mode 1: per row, start of each cell relative to the row
        uint32_t cs[9][MAXLX + 4];
    } tbl;
    Plan plan;
    SysDesc d;      // the system of the current X-row
    float t;        // its kernel scale
    int coarse[9];  // row holds a cell without sub-bin starts: end lookups use cell bounds
    uint32_t row;   // current X-row, local to its system
    int xs, xe;     // its cells [xs, xe) handled by this work item
    int has_row;
    int failed;
    uint64_t bar;
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

// Plans the chunk starting at x0 (warp 0, one pass of global loads): the
// largest x1 such that the chunk has at most TT targets and its 9 source
// rows hold at most CAP particles, plus each row's range.  A single cell
// whose rows exceed CAP is read from global memory (mode 1).
template <int TT, int CAP>
__device__ void plan_chunk(const InteractArgs& a, const SysDesc& d, Plan& p, int x0, int xe, int cy,
                           int cz, unsigned lane)
{
    const int nx = d.g.n[0], ny = d.g.n[1], nz = d.g.n[2];
    const uint32_t cb = d.cell_base;
    const uint32_t rb0 = cb + (uint32_t)nx * ((uint32_t)cy + (uint32_t)ny * (uint32_t)cz);
    const int xa = max(x0 - 1, 0);
    const int xmax = min(xe, x0 + MAXLX);
    // first particle of each row's source range (the same for every lane)
    uint32_t rstart[9];
#pragma unroll
    for (int r = 0; r < 9; ++r) {
        const int by = cy + r % 3 - 1, bz = cz + r / 3 - 1;
        const bool ok = by >= 0 && by < ny && bz >= 0 && bz < nz;
        rstart[r] = ok ? a.offsets[cb + (uint32_t)nx * ((uint32_t)by + (uint32_t)ny * (uint32_t)bz) + xa]
                       : 0u;
    }
    const uint32_t tgt0 = a.offsets[rb0 + x0];
    int best = 0;
    bool first_fits = true;
    for (int base = x0 + 1; base <= xmax; base += 32) {
        const int x1 = base + (int)lane;
        bool valid = false, fits = true;
        if (x1 <= xmax) {
            const int xb = min(x1, nx - 1);
            const uint32_t targets = a.offsets[rb0 + x1] - tgt0;
            uint32_t staged = 0;
#pragma unroll
            for (int r = 0; r < 9; ++r) {
                const int by = cy + r % 3 - 1, bz = cz + r / 3 - 1;
                if (by < 0 || by >= ny || bz < 0 || bz >= nz) continue;
                staged += a.offsets[cb + (uint32_t)nx * ((uint32_t)by + (uint32_t)ny * (uint32_t)bz) + xb + 1] -
                          rstart[r];
            }
            fits = staged <= (uint32_t)CAP;
            valid = fits && targets <= (uint32_t)TT;
        }
        const unsigned vm = __ballot_sync(0xffffffffu, valid);
        if (base == x0 + 1) first_fits = __shfl_sync(0xffffffffu, fits, 0);
        if (vm) best = base + 31 - __clz(vm);
        if (vm != 0xffffffffu) break;
    }
    int x1 = best, mode = 0;
    if (best == 0) {
        x1 = x0 + 1;
        mode = first_fits ? 0 : 1;
    }
    const int xb = min(x1, nx - 1);
    // lane r < 9 owns row r
    uint32_t gb = 0, len = 0;
    if (lane < 9) {
        const int by = cy + (int)lane % 3 - 1, bz = cz + (int)lane / 3 - 1;
        if (by >= 0 && by < ny && bz >= 0 && bz < nz) {
            const uint32_t rb = cb + (uint32_t)nx * ((uint32_t)by + (uint32_t)ny * (uint32_t)bz);
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
        p.gbeg[lane] = gb;
        p.rlen[lane] = (int)len;
        p.sbeg[lane] = (int)(incl - len);
    }
    if (lane == 8) p.total = (int)incl;
    if (lane == 0) {
        p.xa = xa;
        p.xb = xb;
        p.x1 = x1;
        p.mode = mode;
    }
}

// x-bin used by the staged-row lookup: monotone in x (FP32 round-to-nearest
// subtract and multiply, floor), relative to the first source cell xa.
__device__ __forceinline__ int xbin(float x, float lo, float inv4, int base, int nb)
{
    const int b = __float2int_rd(__fmul_rn(__fsub_rn(x, lo), inv4)) - base;
    return min(max(b, 0), nb - 1);
}

// Distances (minus slack, at least 0) from a target to the faces of its own
// cell in y and z; a row offset by dy/dz is at least that far in y/z.
struct Faces {
    float y_lo, y_hi, z_lo, z_hi;
};

__device__ __forceinline__ Faces faces_of(const SysDesc& d, float yt, float zt, int cy, int cz)
{
    const float wy = d.cell_w[1], wz = d.cell_w[2];
    Faces f;
    f.y_lo = fmaxf(yt - fmaf((float)cy, wy, d.g.lo[1]) - d.slack, 0.f);
    f.y_hi = fmaxf(fmaf((float)(cy + 1), wy, d.g.lo[1]) - yt - d.slack, 0.f);
    f.z_lo = fmaxf(zt - fmaf((float)cz, wz, d.g.lo[2]) - d.slack, 0.f);
    f.z_hi = fmaxf(fmaf((float)(cz + 1), wz, d.g.lo[2]) - zt - d.slack, 0.f);
    return f;
}

// Half-width of the x-window of row rr, or a negative value if the row is
// out of reach.  Conservative: rc^2 is inflated by 2e-5 and the slack added.
__device__ __forceinline__ float row_halfwidth(const SysDesc& d, const Faces& f, int rr)
{
    const int dy = rr % 3 - 1, dz = rr / 3 - 1;
    const float ey = dy < 0 ? f.y_lo : (dy > 0 ? f.y_hi : 0.f);
    const float ez = dz < 0 ? f.z_lo : (dz > 0 ? f.z_hi : 0.f);
    const float rcm2 = d.rc2 * 1.00002f;
    const float t = rcm2 - fmaf(ey, ey, ez * ez);
    if (!(t > 0.f)) return -1.f;
    const float tt = fmaxf(t, 1e-30f);
    return tt * rsqrtf(tt) + d.slack;
}

// Two Gaussian candidates at once with packed FP32 (f32x2) arithmetic:
// every element is rounded exactly as the scalar operation would be, so the
// pair test and the sums are those of Sums::pair_nb.
struct PackedSums {
    float2 s = make_float2(0.f, 0.f), vx = make_float2(0.f, 0.f), vy = make_float2(0.f, 0.f),
           vz = make_float2(0.f, 0.f), n = make_float2(0.f, 0.f);

    // second = false drops the second candidate (an odd tail reuses the first)
    __device__ __forceinline__ void pair2(float2 px, float2 py, float2 pz, float2 mx, float2 my,
                                          float2 mz, float rc2, float2 ks, bool second = true)
    {
        const float2 dx = __fadd2_rn(px, mx);
        const float2 dy = __fadd2_rn(py, my);
        const float2 dz = __fadd2_rn(pz, mz);
        const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
        const float2 t = __fmul2_rn(r2, ks);
        const bool i0 = r2.x < rc2, i1 = (r2.y < rc2) && second;
        const float e0 = ex2_approx(t.x), e1 = ex2_approx(t.y);
        const float2 K = make_float2(i0 ? e0 : 0.f, i1 ? e1 : 0.f);
        s = __fadd2_rn(s, K);
        vx = __ffma2_rn(dx, K, vx);
        vy = __ffma2_rn(dy, K, vy);
        vz = __ffma2_rn(dz, K, vz);
        n = __fadd2_rn(n, make_float2(i0 ? 1.f : 0.f, i1 ? 1.f : 0.f));
    }
};

// The candidates [j, je) of one row window, in order.  The Gaussian FP32
// path takes them two at a time (packed, even and odd partial sums); the
// others one at a time.  Shared by the staged and the global-memory paths so
// that both sum every target's terms in the same order.
template <class Acc, int KERNEL>
__device__ __forceinline__ void window_sums(const float4* src, int j, int je, float xt, float yt,
                                            float zt, uint32_t slot, float rc2, const KParams& kp,
                                            PackedSums& ps, Sums<Acc, KERNEL>& r)
{
    constexpr bool packed = std::is_same<Acc, PlainAcc>::value && KERNEL == KERNEL_GAUSSIAN;
    constexpr bool by_id = self_by_identity<KERNEL, Acc>();
    if constexpr (packed) {
        const float2 mx = make_float2(-xt, -xt), my = make_float2(-yt, -yt), mz = make_float2(-zt, -zt),
                     ks = make_float2(kp.t, kp.t);
        for (; j < je; j += 2) {
            const bool two = j + 1 < je;
            const float4 s0 = src[j], s1 = src[two ? j + 1 : j];
            ps.pair2(make_float2(s0.x, s1.x), make_float2(s0.y, s1.y), make_float2(s0.z, s1.z), mx, my,
                     mz, rc2, ks, two);
        }
    } else {
        for (; j < je; ++j) {
            const float4 s0 = src[j];
            r.pair_nb(__fsub_rn(s0.x, xt), __fsub_rn(s0.y, yt), __fsub_rn(s0.z, zt), rc2, kp,
                      by_id && __float_as_uint(s0.w) == slot);
        }
    }
}

template <class Acc, int KERNEL>
__device__ __forceinline__ void finish_packed(const PackedSums& ps, Sums<Acc, KERNEL>& r)
{
    if constexpr (std::is_same<Acc, PlainAcc>::value && KERNEL == KERNEL_GAUSSIAN) {
        r.s.add(ps.s.x + ps.s.y);
        r.vx.add(ps.vx.x + ps.vx.y);
        r.vy.add(ps.vy.x + ps.vy.y);
        r.vz.add(ps.vz.x + ps.vz.y);
        r.n += (uint32_t)(ps.n.x + ps.n.y);
    }
}

// Global-memory path (mode 1) for one target: per row, the window
// [first x >= x - w, first x > x + w) by binary search inside the cells of
// x - w and x + w, summed exactly as the staged path does.
template <class Acc, int KERNEL, class SM>
__device__ __forceinline__ void target_sums_global(const InteractArgs& a, const SM& sm, float xt,
                                                   float yt, float zt, uint32_t slot, int cy, int cz,
                                                   const KParams& kp, Sums<Acc, KERNEL>& r)
{
    const Plan& p = sm.plan;
    const SysDesc& d = sm.d;
    const Faces f = faces_of(d, yt, zt, cy, cz);
    PackedSums ps;
#pragma unroll 1
    for (int rr = 0; rr < 9; ++rr) {
        const int len = p.rlen[rr];
        if (len == 0) continue;
        const float w = row_halfwidth(d, f, rr);
        if (w < 0.f) continue;
        const float xlo = xt - w, xhi = xt + w;
        const int kmax = p.xb - p.xa;
        const int k0 = min(max(axis_cell(xlo, d.g.lo[0], d.g.inv_w[0], d.g.n[0]) - p.xa, 0), kmax);
        const int k1 = min(max(axis_cell(xhi, d.g.lo[0], d.g.inv_w[0], d.g.n[0]) - p.xa, 0), kmax);
        const float4* row = a.P + p.gbeg[rr];
        int lo = (int)sm.tbl.cs[rr][k0], hi = (int)sm.tbl.cs[rr][k0 + 1];
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (row[mid].x < xlo) lo = mid + 1;
            else hi = mid;
        }
        int e0 = max((int)sm.tbl.cs[rr][k1], lo), e1 = (int)sm.tbl.cs[rr][k1 + 1];
        while (e0 < e1) {
            const int mid = (e0 + e1) >> 1;
            if (row[mid].x > xhi) e1 = mid;
            else e0 = mid + 1;
        }
        window_sums<Acc, KERNEL>(row, lo, e0, xt, yt, zt, slot, d.rc2, kp, ps, r);
    }
    finish_packed(ps, r);
}

// Sums of one target over the staged rows (mode 0).  Per row: the x-window
// from the row's lookup table, trimmed to [x - w, x + w] exactly; every
// source in it is a candidate, taken two at a time.
template <class Acc, int KERNEL, class SM>
__device__ __forceinline__ void target_sums_staged(const SM& sm, float xt, float yt, float zt,
                                                   uint32_t slot, int cy, int cz, int ncell,
                                                   float inv4, const KParams& kp,
                                                   Sums<Acc, KERNEL>& r)
{
    const Plan& p = sm.plan;
    const SysDesc& d = sm.d;
    const Faces f = faces_of(d, yt, zt, cy, cz);
    const int nb = ncell * BPC, base = BPC * p.xa;
    PackedSums ps;
#pragma unroll 1
    for (int rr = 0; rr < 9; ++rr) {
        if (p.rlen[rr] == 0) continue;
        const float w = row_halfwidth(d, f, rr);
        if (w < 0.f) continue;
        const float xlo = xt - w, xhi = xt + w;
        int j = sm.tbl.bin[rr][xbin(xlo, d.g.lo[0], inv4, base, nb)];
        int bh = xbin(xhi, d.g.lo[0], inv4, base, nb) + 1;
        if (sm.coarse[rr]) bh = (bh + BPC - 1) / BPC * BPC;
        int je = sm.tbl.bin[rr][bh];
        while (j < je && sm.buf[j].x < xlo) ++j;
        while (je > j && sm.buf[je - 1].x > xhi) --je;
        // window [j, je): every source in it is a candidate
        window_sums<Acc, KERNEL>(sm.buf, j, je, xt, yt, zt, slot, d.rc2, kp, ps, r);
    }
    finish_packed(ps, r);
}

template <class T, class Acc, int KERNEL>
__global__ void __launch_bounds__(T::TT, T::MINB) k_interact_tiled(InteractArgs a)
{
    constexpr int TT = T::TT, CAP = T::CAP;
    __shared__ Smem<CAP> sm;

    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctrl->work[(a.seq + 1u) & 1u] = 0u;
    if (load_error(a.ctrl)) return;
    const unsigned tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    // The self pair (r = 0) adds exactly kernel_value(0) to S and 1 to n;
    // both are taken off at the end instead of testing identities per pair
    // (except for the kernels of self_by_identity).
    const float k0_scale_free = KERNEL == KERNEL_GAUSSIAN ? ex2_approx(0.f) : 0.f;

    if (tid == 0) {
        sm.failed = 0;
        bar_init(&sm.bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t phase = 0;

    for (;;) {
        if (tid == 0) {
            const uint32_t item = atomicAdd(&a.ctrl->work[a.seq & 1u], 1u);
            sm.has_row = item < a.work;
            if (item < a.work) {
                const int sid = a.sy.S == 1 ? 0 : find_system(a.sy.wbase, a.sy.S, item);
                sm.d = a.sy.sys[sid];
                sm.t = a.kscale ? a.kscale[sid] : a.kscale0;
                const uint32_t local = item - sm.d.work_base;
                const uint32_t seg = local % sm.d.nseg;
                sm.row = local / sm.d.nseg;
                sm.xs = (int)seg * SEG_CELLS;
                sm.xe = min(sm.d.g.n[0], (int)(seg + 1) * SEG_CELLS);
            }
        }
        __syncthreads();
        if (!sm.has_row || sm.failed) break;
        const uint32_t row = sm.row;
        const SysDesc& d = sm.d;
        const int nx = d.g.n[0], ny = d.g.n[1];
        const float inv4 = d.g.inv_w[0] * (float)BPC;
        const int cy = (int)(row % (uint32_t)ny), cz = (int)(row / (uint32_t)ny);
        const uint32_t rb0 = d.cell_base + (uint32_t)nx * row;
        // the self pair's contribution (0 where it is excluded by identity)
        float kself = k0_scale_free;
        uint32_t nself = 1u;
        if constexpr (KERNEL == KERNEL_LOWFLOP) kself = 1.0f;
        if constexpr (self_by_identity<KERNEL, Acc>()) {
            kself = 0.f;
            nself = 0u;
        }

        const int xe = sm.xe;
        for (int x0 = sm.xs; x0 < xe;) {
            if (warp == 0) {
                if (lane < 9) sm.coarse[lane] = 0;
                plan_chunk<TT, CAP>(a, d, sm.plan, x0, xe, cy, cz, lane);
                __syncwarp();
                if (lane == 0 && sm.plan.mode == 0) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    bar_expect_tx(&sm.bar, (uint32_t)sm.plan.total * 16u);
                    for (int rr = 0; rr < 9; ++rr)
                        if (sm.plan.rlen[rr] > 0)
                            bulk_g2s(&sm.buf[sm.plan.sbeg[rr]], a.P + sm.plan.gbeg[rr],
                                     (uint32_t)sm.plan.rlen[rr] * 16u, &sm.bar);
                }
            }
            __syncthreads();
            const Plan& p = sm.plan;
            const int x1 = p.x1, mode = p.mode, xa = p.xa;
            const int ncell = p.xb - xa + 1;
            // Row lookup tables, built from the offsets and the per-cell
            // sub-bin starts while the bulk copies are in flight.
            for (int e = tid; e < 9 * (ncell + 1); e += TT) {
                const int rr = e / (ncell + 1), k = e % (ncell + 1);
                if (p.rlen[rr] == 0) continue;
                const int by = cy + rr % 3 - 1, bz = cz + rr / 3 - 1;
                const uint32_t cidx =
                    d.cell_base + (uint32_t)nx * ((uint32_t)by + (uint32_t)ny * (uint32_t)bz) + xa + k;
                const uint32_t g = a.offsets[cidx];
                if (mode == 0) {
                    const int start = p.sbeg[rr] + (int)(g - p.gbeg[rr]);
                    if (k == ncell) {
                        sm.tbl.bin[rr][BPC * ncell] = (uint16_t)start;
                    } else {
                        const uint32_t w = a.xbins[cidx];
                        if (w >> 24) sm.coarse[rr] = 1;
                        sm.tbl.bin[rr][BPC * k] = (uint16_t)start;
                        sm.tbl.bin[rr][BPC * k + 1] = (uint16_t)(start + (int)(w & 255u));
                        sm.tbl.bin[rr][BPC * k + 2] = (uint16_t)(start + (int)((w >> 8) & 255u));
                        sm.tbl.bin[rr][BPC * k + 3] = (uint16_t)(start + (int)((w >> 16) & 255u));
                    }
                } else {
                    sm.tbl.cs[rr][k] = g - p.gbeg[rr];
                }
            }
            if (mode == 0) {
                if (!bar_wait_bounded(&sm.bar, phase, a.wait_limit_ns)) {
                    sm.failed = 1;
                    atomicOr(&a.ctrl->error, ERR_TIMEOUT);
                    // let the copies in flight land before the CTA exits
                    bar_wait_bounded(&sm.bar, phase, a.wait_limit_ns);
                }
                phase ^= 1u;
            }
            __syncthreads();  // tables ready; sm.failed is uniform from here on
            const uint32_t tb = a.offsets[rb0 + x0], te = a.offsets[rb0 + x1];
            const int ntarget = (int)(te - tb);
            // staged index of the first target (the centre row is row 4)
            const int t0 = p.sbeg[4] + (int)(tb - p.gbeg[4]);
            if (!sm.failed) {
                for (int q0 = 0; q0 < ntarget; q0 += TT) {
                    const int q = q0 + (int)tid;
                    if (q >= ntarget) continue;
                    Sums<Acc, KERNEL> r;
                    const KParams kp{sm.t, a.one, a.zero};
                    const float4 me = mode == 0 ? sm.buf[t0 + q] : a.P[tb + q];
                    const uint32_t slot = __float_as_uint(me.w);
                    if (mode == 0)
                        target_sums_staged<Acc, KERNEL>(sm, me.x, me.y, me.z, slot, cy, cz, ncell, inv4,
                                                        kp, r);
                    else
                        target_sums_global<Acc, KERNEL>(a, sm, me.x, me.y, me.z, slot, cy, cz, kp, r);
                    store_out(a, slot, r, kself, nself);
                }
            }
            __syncthreads();
            x0 = x1;
        }
    }
}

template <class Acc>
cudaError_t launch_ppnl_acc(const InteractArgs& a, cudaStream_t s)
{
    const unsigned blocks = (unsigned)((a.n + 127) / 128);
    switch (a.kernel) {
        case KERNEL_LJ: k_interact_ppnl<Acc, KERNEL_LJ><<<blocks, 128, 0, s>>>(a); break;
        case KERNEL_LOWFLOP: k_interact_ppnl<Acc, KERNEL_LOWFLOP><<<blocks, 128, 0, s>>>(a); break;
        case KERNEL_HIGHFLOP: k_interact_ppnl<Acc, KERNEL_HIGHFLOP><<<blocks, 128, 0, s>>>(a); break;
        default: k_interact_ppnl<Acc, KERNEL_GAUSSIAN><<<blocks, 128, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

template <class Acc>
cudaError_t launch_tiled_acc(const InteractArgs& a, int tile, const int* per_sm, int num_sms,
                             cudaStream_t s)
{
    // the other kernels are comparators: they run with the middle tile shape
    if (a.kernel != KERNEL_GAUSSIAN) tile = 1;
    const int TTs[3] = {Tile64::TT, Tile128::TT, Tile256::TT};
    uint64_t grid = (uint64_t)num_sms * (uint64_t)(per_sm[tile] < 1 ? 1 : per_sm[tile]);
    if (grid > a.work) grid = a.work;
    if (grid < 1) grid = 1;
    const unsigned g = (unsigned)grid;
    const int tt = TTs[tile];
    switch (a.kernel) {
        case KERNEL_LJ: k_interact_tiled<Tile128, Acc, KERNEL_LJ><<<g, tt, 0, s>>>(a); break;
        case KERNEL_LOWFLOP: k_interact_tiled<Tile128, Acc, KERNEL_LOWFLOP><<<g, tt, 0, s>>>(a); break;
        case KERNEL_HIGHFLOP: k_interact_tiled<Tile128, Acc, KERNEL_HIGHFLOP><<<g, tt, 0, s>>>(a); break;
        default:
            if (tile == 0) k_interact_tiled<Tile64, Acc, KERNEL_GAUSSIAN><<<g, tt, 0, s>>>(a);
            else if (tile == 2) k_interact_tiled<Tile256, Acc, KERNEL_GAUSSIAN><<<g, tt, 0, s>>>(a);
            else k_interact_tiled<Tile128, Acc, KERNEL_GAUSSIAN><<<g, tt, 0, s>>>(a);
            break;
    }
    return cudaGetLastError();
}

template <class T, class Acc>
cudaError_t occupancy_of(int* per_sm)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_interact_tiled<T, Acc, KERNEL_GAUSSIAN>,
                                                         T::TT, 0);
}

}  // namespace

cudaError_t launch_interact_ppnl(const InteractArgs& a, bool kahan, int num_sms, cudaStream_t s,
                                 int* launches)
{
    (void)num_sms;
    *launches += 1;
    return kahan ? launch_ppnl_acc<KahanAcc>(a, s) : launch_ppnl_acc<PlainAcc>(a, s);
}

cudaError_t tiled_occupancy(bool kahan, int* per_sm)
{
    cudaError_t e;
    if (kahan) {
        if ((e = occupancy_of<Tile64, KahanAcc>(&per_sm[0])) != cudaSuccess) return e;
        if ((e = occupancy_of<Tile128, KahanAcc>(&per_sm[1])) != cudaSuccess) return e;
        return occupancy_of<Tile256, KahanAcc>(&per_sm[2]);
    }
    if ((e = occupancy_of<Tile64, PlainAcc>(&per_sm[0])) != cudaSuccess) return e;
    if ((e = occupancy_of<Tile128, PlainAcc>(&per_sm[1])) != cudaSuccess) return e;
    return occupancy_of<Tile256, PlainAcc>(&per_sm[2]);
}

cudaError_t launch_interact_tiled(const InteractArgs& a, bool kahan, int num_sms, const int* per_sm,
                                  int tile, cudaStream_t s, int* launches)
{
    *launches += 1;
    return kahan ? launch_tiled_acc<KahanAcc>(a, tile, per_sm, num_sms, s)
                 : launch_tiled_acc<PlainAcc>(a, tile, per_sm, num_sms, s);
}

}  // namespace pi
