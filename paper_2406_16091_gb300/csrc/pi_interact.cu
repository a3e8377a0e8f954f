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
//   k_interact_ppnl    Alg. 1 (Par-Part-NoLoop): one thread per particle,
//                      sources read straight from global memory.  Kept as
//                      the comparator the paper measures its speedups
//                      against.
// The others read P, the x-ordered copy written by binning: the sorted
// particles as float4 (x, y, z, stable slot), every X-row of cells sorted by
// x as a whole and followed by ROW_PADS sentinel slots.  A target scans, per
// neighbour row (y +- 1, z +- 1), only the x-window [x_i - w_r, x_i + w_r],
// w_r = sqrt(rc^2 - d_yz^2) with d_yz its distance to the row in y and z
// (sources outside it cannot pass the pair test), found from per-cell
// x-sub-bin starts; each thread takes two x-adjacent targets and evaluates
// every source against both with packed f32x2 arithmetic.
//   k_interact_direct  (default) one thread per target pair, windows from
//                      global memory, sources read through L1; one flattened
//                      loop over all windows.  Every kernel K and both
//                      precision modes.
//   k_interact_tiled   work items are segments of an X-row of target cells,
//                      handed out dynamically from one queue over all
//                      systems and processed in chunks of consecutive cells;
//                      the 9 neighbour rows of a chunk are contiguous ranges
//                      of P, each staged into shared memory with one
//                      cp.async.bulk copy (Sec. 5.2 loads pencils along X;
//                      here the whole 3x3 bundle is loaded at once because
//                      the sorted order makes each one contiguous).
//   k_interact_ws      the same chunks with a producer warp that stages them
//                      for consumer warps (warp specialisation).
// All of them sum each target's terms in the order of its own windows, so
// their outputs are bitwise equal.  Every one is a programmatic dependent
// launch: it may start while the binning's last kernel (or the previous
// interaction) drains, and waits for it before reading anything of the step.
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

// Accumulators.  add(t, in) adds the term t of a candidate that passed the
// pair test (in) or the exact zero of one that did not (!in); both leave the
// sum exactly as it was for a zero, so that candidates outside a target's
// own windows never change its sums.
struct PlainAcc {
    float v = 0.f;
    __device__ __forceinline__ void add(float t, bool) { v = __fadd_rn(v, t); }
    __device__ __forceinline__ void addmul(float a, float b, bool) { v = __fmaf_rn(a, b, v); }
    __device__ __forceinline__ float value() const { return v; }
};

// Kahan-compensated FP32 accumulation (precision mode).  A rejected
// candidate is skipped altogether: a compensated add of zero would fold the
// pending compensation into the sum, making the result depend on how many
// rejected candidates a path reads.
struct KahanAcc {
    float v = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float t, bool in)
    {
        const float y = __fsub_rn(t, c);
        const float u = __fadd_rn(v, y);
        const float c1 = __fsub_rn(__fsub_rn(u, v), y);
        v = in ? u : v;
        c = in ? c1 : c;
    }
    __device__ __forceinline__ void addmul(float a, float b, bool in) { add(__fmul_rn(a, b), in); }
    __device__ __forceinline__ float value() const { return v; }
};

// Scale of the kernel (t; for the fine Gaussian also the remainder tl of
// the FP64 scale after t) and the opaque constants of the high-FLOP kernel.
struct KParams {
    float t, tl, one, zero;
};

// s + e = a + b exactly (Knuth's two-sum, six rounded operations).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

constexpr float LN2_F = 0.693147180559945309f;

// exp(-r^2/h^2) for a short kernel length h.  In FP32 the exponent
// u = r2 t carries the rounding of r2 and of t relative to |u|, which reaches
// 64 log2(e) at h = r_c/8, so the plain form's relative error per term grows
// as (r/h)^2 (about 1e-5 at h = r_c/10).  Here r^2 of the FP32 offsets is
// kept as a sum with its rounding errors (exact squares by fma, two-sums),
// the product with the scale t + tl keeps its rounding error (fma), and the
// small remainder c of the exponent is applied to first order:
// K = 2^uh (1 + c ln 2), accurate to a few ulp whatever h.  For a far
// candidate (a row's sentinel slots at 1e18) uh overflows to -inf and c to
// +inf or NaN; c is clamped to [-1, 1] (fminf/fmaxf return the number
// against a NaN) so that K = 0 * (1 + c ln 2) stays an exact 0, which the
// pair test's mask then keeps out of the sums.
__device__ __forceinline__ float gauss_fine(float dx, float dy, float dz, float th, float tl)
{
    const float px = __fmul_rn(dx, dx), ex = __fmaf_rn(dx, dx, -px);
    const float py = __fmul_rn(dy, dy), ey = __fmaf_rn(dy, dy, -py);
    const float pz = __fmul_rn(dz, dz), ez = __fmaf_rn(dz, dz, -pz);
    float s1, e1, s2, e2;
    two_sum(px, py, s1, e1);
    two_sum(s1, pz, s2, e2);
    const float uh = __fmul_rn(s2, th);
    const float ue = __fmaf_rn(s2, th, -uh);
    const float es = __fadd_rn(__fadd_rn(ex, ey), __fadd_rn(ez, __fadd_rn(e1, e2)));
    const float c = fminf(fmaxf(__fmaf_rn(th, es, __fmaf_rn(tl, s2, ue)), -1.f), 1.f);
    const float k0 = ex2_approx(uh);
    return __fmaf_rn(__fmul_rn(k0, c), LN2_F, k0);
}

// Value of the interaction kernel for one pair inside the cutoff at FP32
// offset (dx, dy, dz), r2 the frozen FP32 squared distance; kp.t is the
// system's scale (Gaussian: -log2(e)/h^2; Lennard-Jones: sigma^2).
template <int KERNEL>
__device__ __forceinline__ float kernel_value(float dx, float dy, float dz, float r2, const KParams& kp)
{
    if constexpr (KERNEL == KERNEL_GAUSSIAN) {
        return ex2_approx(__fmul_rn(r2, kp.t));
    } else if constexpr (KERNEL == KERNEL_GAUSSIAN_FINE) {
        return gauss_fine(dx, dy, dz, kp.t, kp.tl);
    } else if constexpr (KERNEL == KERNEL_LOWFLOP) {
        return 1.0f;
    } else {
        const float t = kp.t;
        const float rs2 = __fmaf_rn(0.01f, t, r2);
        const float sr = __fmul_rn(t, __frcp_rn(rs2));
        const float s3 = __fmul_rn(__fmul_rn(sr, sr), sr);
        float K = __fmul_rn(4.0f, __fsub_rn(__fmul_rn(s3, s3), s3));
        if constexpr (KERNEL == KERNEL_HIGHFLOP) {
#pragma unroll
            for (int i = 0; i < 75; ++i) K = __fmaf_rn(K, kp.one, kp.zero);
        }
        return K;
    }
}

// The kernel parameters of system sid: kscale holds the S scales, then the
// S remainders of the fine Gaussian.
__device__ __forceinline__ KParams kparams(const InteractArgs& a, int sid)
{
    return a.kscale ? KParams{a.kscale[sid], a.kscale[a.sy.S + sid], a.one, a.zero}
                    : KParams{a.kscale0, a.kscale0_lo, a.one, a.zero};
}

// Every path excludes the self pair by identity (the source's stable slot
// equals the target's), as Sec. 2's j != i states: adding K(0) and taking it
// off at the end would round every partial sum at the magnitude of K(0),
// which for a short kernel length h is far larger than the particle's sum.

// Per-target accumulators of one interaction kernel.
template <class Acc, int KERNEL>
struct Sums {
    Acc s, vx, vy, vz;
    uint32_t n = 0;

    __device__ __forceinline__ void add(float dx, float dy, float dz, float K, bool in)
    {
        s.add(K, in);
        vx.addmul(dx, K, in);
        vy.addmul(dy, K, in);
        vz.addmul(dz, K, in);
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
        const float e = kernel_value<KERNEL>(dx, dy, dz, r2, kp);
        add(dx, dy, dz, in ? e : 0.f, in);
    }

    // One candidate source at FP32 offset (dx, dy, dz) from the target.
    __device__ __forceinline__ void pair(float dx, float dy, float dz, float rc2, const KParams& kp)
    {
        const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
        if (r2 < rc2) add(dx, dy, dz, kernel_value<KERNEL>(dx, dy, dz, r2, kp), true);
    }
};

template <class Acc, int KERNEL>
__device__ __forceinline__ void store_out(const InteractArgs& a, uint32_t slot, const Sums<Acc, KERNEL>& r)
{
    if (!PI_BOUNDS(a.ctrl, slot, a.n, CS_DIRECT_TARGET)) return;
    const uint32_t o = a.original_order ? a.perm[slot] : slot;
    if (!PI_BOUNDS(a.ctrl, o, a.n, CS_DIRECT_TARGET)) return;
    a.S[o] = r.s.value();
    a.Vx[o] = r.vx.value();
    a.Vy[o] = r.vy.value();
    a.Vz[o] = r.vz.value();
    if (a.nbr) a.nbr[o] = r.n;
}

// ---- Alg. 1: Par-Part-NoLoop ------------------------------------------------

template <class Acc, int KERNEL>
__global__ void __launch_bounds__(128) k_interact_ppnl(InteractArgs a)
{
    pdl_trigger();
    pdl_wait();
    if (cta_error(a.ctrl)) return;
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
    const KParams kp = kparams(a, sid);
    for (int bz = max(cz - 1, 0); bz <= min(cz + 1, nz - 1); ++bz)
        for (int by = max(cy - 1, 0); by <= min(cy + 1, ny - 1); ++by) {
            const uint32_t row = d.cell_base + (uint32_t)nx * ((uint32_t)by + (uint32_t)ny * (uint32_t)bz);
            const uint32_t j0 = a.offsets[row + max(cx - 1, 0)];
            const uint32_t j1 = a.offsets[row + min(cx + 1, nx - 1) + 1];
            if (!PI_BOUNDS(a.ctrl, j1, (uint64_t)a.n + 1u, CS_PPNL_SRC)) continue;
            for (uint32_t j = j0; j < j1; ++j) {
                if (j == k) continue;
                r.pair(__fsub_rn(a.sx[j], xt), __fsub_rn(a.sy_pos[j], yt), __fsub_rn(a.sz[j], zt), d.rc2, kp);
            }
        }
    store_out(a, k, r);
}

// ---- tiled interaction ----------------------------------------------------------

// Tile shapes of the one-CTA-per-chunk kernel: threads per CTA (each takes
// two targets, so a chunk has up to 2 NT targets), staged particles per
// chunk, CTAs per SM the register and shared-memory budget is sized for, and
// target cells per chunk along X.  The autotuner (pi_autotune) picks one per
// context; every shape gives the same per-target summation order, so the
// results are identical.
template <int NT_, int CAP_, int MINB_, int MAXLX_>
struct Tile {
    static constexpr int NT = NT_;
    static constexpr int TT = 2 * NT_;  // most targets per chunk (planner limit)
    static constexpr int CAP = CAP_;
    static constexpr int MINB = MINB_;
    static constexpr int MAXLX = MAXLX_;
    // lookup-table entries per row: XSUB per source cell plus the row end,
    // rounded up so that every row starts 16-byte aligned
    static constexpr int RB = ((MAXLX + 2) * XSUB + 1 + 7) / 8 * 8;
};
using TileS = Tile<32, 768, 12, 16>;
using TileM = Tile<64, 1280, 7, SEG_CELLS>;
using TileL = Tile<128, 2432, 4, SEG_CELLS>;

// Sentinel slots staged after every row: the window loop reads whole groups
// of four candidates, and up to three slots past a window's end are either
// particles of the same row outside the window or these sentinels; the
// pair test rejects both.
constexpr int ROW_PAD = 3;

// Lookup-table entries per row of a chunk read from global memory (mode 1:
// one target cell, so at most 3 source cells).
constexpr int RB_GLOBAL = 3 * XSUB + 1;

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
    int total;  // staged particles (without the sentinel slots)
};

template <class T>
struct Smem {
    // Staged rows.  buf[CAP] is a sentinel far from every particle: an odd
    // tail pairs its last candidate with it, and the pair test rejects it.
    float4 buf[T::CAP + 1];
    // Per row r and sub-bin b of the chunk's source cells (b = XSUB * cell +
    // sub-bin, counted from cell xa): index of the first particle of row r
    // whose sub-bin is >= b; entry XSUB * ncell is the row end.  Staged
    // indices in mode 0, indices into P in mode 1.
    union {
        __align__(16) uint16_t staged[9][T::RB];
        uint32_t global[9][RB_GLOBAL];
    } tbl;
    // Per thread: the non-empty x-windows of its targets as byte offsets
    // into buf, first | end << 16, plus one spare row read after the last.
    uint32_t win[10][T::NT];
    Plan plan;
    SysDesc d;             // the system of the current X-row
    KParams kp;            // its kernel parameters
    uint32_t coarse_mask;  // bit r: row r holds a cell without sub-bin starts
    uint32_t row;          // current X-row, local to its system
    int xs, xe;            // its cells [xs, xe) handled by this work item
    int has_row;
    int failed;
    uint64_t bar;
};

// MINB CTAs of a shape fit the SM's 228 KB of shared memory (1 KB of which
// each CTA reserves).
template <class T>
constexpr bool fits_sm()
{
    return T::MINB * (sizeof(Smem<T>) + 1024) <= 228u * 1024u;
}
static_assert(fits_sm<TileS>() && fits_sm<TileM>() && fits_sm<TileL>(),
              "tile shapes exceed the shared memory of their CTAs per SM");

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Two consecutive float4s from a 32-byte aligned global address, as one
// 256-bit read-only vector load.
__device__ __forceinline__ void ldg_pair(const float4* q, float4& u, float4& v)
{
    unsigned long long a0, a1, a2, a3;
    asm("ld.global.nc.v4.b64 {%0, %1, %2, %3}, [%4];" : "=l"(a0), "=l"(a1), "=l"(a2), "=l"(a3) : "l"(q));
    u = make_float4(__uint_as_float((uint32_t)a0), __uint_as_float((uint32_t)(a0 >> 32)),
                    __uint_as_float((uint32_t)a1), __uint_as_float((uint32_t)(a1 >> 32)));
    v = make_float4(__uint_as_float((uint32_t)a2), __uint_as_float((uint32_t)(a2 >> 32)),
                    __uint_as_float((uint32_t)a3), __uint_as_float((uint32_t)(a3 >> 32)));
}

// Shared-memory loads by 32-bit shared-window address.  The "memory"
// clobber keeps them after the C++ stores that wrote the data.
__device__ __forceinline__ float4 lds_f4(uint32_t addr)
{
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr)
                 : "memory");
    return v;
}

__device__ __forceinline__ uint32_t lds_u32(uint32_t addr)
{
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
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
template <class T>
__device__ void plan_chunk(const InteractArgs& a, const SysDesc& d, Plan& p, int x0, int xe, int cy,
                           int cz, unsigned lane)
{
    const int nx = d.g.n[0], ny = d.g.n[1], nz = d.g.n[2];
    const uint32_t cb = d.cell_base;
    const uint32_t rb0 = cb + (uint32_t)nx * ((uint32_t)cy + (uint32_t)ny * (uint32_t)cz);
    const int xa = max(x0 - 1, 0);
    const int xmax = min(xe, x0 + T::MAXLX);
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
            fits = staged + 9u * ROW_PAD <= (uint32_t)T::CAP;
            valid = fits && targets <= (uint32_t)T::TT;
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
            const uint32_t row = (uint32_t)by + (uint32_t)ny * (uint32_t)bz;
            const uint32_t rb = cb + (uint32_t)nx * row;
            const uint32_t s0 = a.offsets[rb + xa];
            len = a.offsets[rb + xb + 1] - s0;
            gb = s0 + ROW_PADS * (d.row_base + row);  // P index
        }
    }
    // staged rows follow each other with ROW_PAD sentinel slots after each
    const uint32_t slots = lane < 9 ? len + ROW_PAD : 0u;
    uint32_t incl = slots, tot = len;
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        const uint32_t u = __shfl_up_sync(0xffffffffu, tot, o);
        if (lane >= (unsigned)o) {
            incl += v;
            tot += u;
        }
    }
    if (lane < 9) {
        p.gbeg[lane] = gb;
        p.rlen[lane] = (int)len;
        p.sbeg[lane] = (int)(incl - slots);
    }
    if (lane == 8) p.total = (int)tot;
    if (lane == 0) {
        p.xa = xa;
        p.xb = xb;
        p.x1 = x1;
        p.mode = mode;
    }
}

// A particle far from every other one (finite coordinates, so its pair
// terms are exact zeros).
__device__ __forceinline__ float4 sentinel()
{
    return make_float4(1e18f, 1e18f, 1e18f, __uint_as_float(0xffffffffu));
}

// The sentinel slots after the staged rows of a chunk (one warp).
template <int CAP>
__device__ __forceinline__ void write_row_pads(float4* buf, const Plan& p, unsigned lane, Ctrl* ctrl)
{
    if (lane < 9u * ROW_PAD) {
        const int rr = (int)lane / ROW_PAD;
        const int at = p.sbeg[rr] + p.rlen[rr] + (int)lane % ROW_PAD;
        if (PI_BOUNDS(ctrl, at, CAP, CS_STAGED_BUF)) buf[at] = sentinel();
    }
    (void)ctrl;
}

// Whether the staged rows of a plan fit the buffer (debug builds; always
// true otherwise: plan_chunk sizes mode-0 chunks to CAP).
template <int CAP>
__device__ __forceinline__ bool rows_fit(const Plan& p, Ctrl* ctrl)
{
    bool ok = true;
#ifdef PI_CHECK
    for (int rr = 0; rr < 9; ++rr) ok = ok && PI_BOUNDS(ctrl, p.sbeg[rr] + p.rlen[rr], CAP + 1, CS_STAGED_BUF);
#endif
    (void)p;
    (void)ctrl;
    return ok;
}

// Lookup table of one chunk, built from the offsets and the per-cell
// sub-bin starts (no staged data needed, so it overlaps the bulk copies).
// The NT threads share the (row, cell) items; every thread first issues the
// loads of all its items, then writes them, so the loads overlap.  Rows
// without particles (or outside the grid) get all-zero entries, i.e. empty
// windows.
template <int NT, class E, int RB>
__device__ __forceinline__ void build_table(const InteractArgs& a, const SysDesc& d, const Plan& p,
                                            int cy, int cz, int ncell, E (*tbl)[RB],
                                            uint32_t* coarse_mask, unsigned t)
{
    constexpr int MAXC = RB / XSUB + 1;              // bound of ncell + 1
    constexpr int MAXI = (9 * MAXC + NT - 1) / NT;   // items per thread
    const int nx = d.g.n[0], ny = d.g.n[1];
    const int per = ncell + 1, total = 9 * per;
    const float inv = 1.0f / (float)per;
    uint32_t start[MAXI];
    uint2 w[MAXI];
#pragma unroll
    for (int i = 0; i < MAXI; ++i) {
        const int e = (int)t + i * NT;
        // e / per in FP32: (e + 1/2) / per is at least 1/(2 per) from an integer
        const int rr = (int)(((float)e + 0.5f) * inv), k = e - rr * per;
        start[i] = 0u;
        w[i] = make_uint2(0u, 0u);
        if (e < total && p.rlen[rr] > 0) {
            const int by = cy + rr % 3 - 1, bz = cz + rr / 3 - 1;
            const uint32_t row = (uint32_t)by + (uint32_t)ny * (uint32_t)bz;
            const uint32_t cidx = d.cell_base + (uint32_t)nx * row + p.xa + k;
            // mode 0: staged index = sbeg + (P index - gbeg); mode 1: P index
            const uint32_t shift = ROW_PADS * (d.row_base + row) +
                                   (sizeof(E) == 2 ? (uint32_t)p.sbeg[rr] - p.gbeg[rr] : 0u);
            start[i] = a.offsets[cidx] + shift;
            if (k < ncell) w[i] = a.xbins[cidx];
        }
    }
#pragma unroll
    for (int i = 0; i < MAXI; ++i) {
        const int e = (int)t + i * NT;
        if (e >= total) break;
        const int rr = (int)(((float)e + 0.5f) * inv), k = e - rr * per;
        if (!PI_BOUNDS(a.ctrl, XSUB * k + (k == ncell ? 1 : XSUB), RB + 1, CS_STAGED_TABLE)) continue;
        E* ent = &tbl[rr][XSUB * k];
        if (k == ncell) {
            ent[0] = (E)start[i];
            continue;
        }
        if ((w[i].y >> 24) & XBIN_COARSE) atomicOr(coarse_mask, 1u << rr);
        E v[XSUB];
        v[0] = (E)start[i];
#pragma unroll
        for (int b = 1; b < XSUB; ++b) {
            const uint32_t word = b <= 4 ? w[i].x : w[i].y;
            v[b] = (E)(start[i] + ((word >> (8 * ((b - 1) & 3))) & 255u));
        }
        if constexpr (sizeof(E) == 2) {
            static_assert(XSUB == 8 && RB % 8 == 0, "one 16-byte store per cell");
            uint4 q;
            q.x = (uint32_t)v[0] | ((uint32_t)v[1] << 16);
            q.y = (uint32_t)v[2] | ((uint32_t)v[3] << 16);
            q.z = (uint32_t)v[4] | ((uint32_t)v[5] << 16);
            q.w = (uint32_t)v[6] | ((uint32_t)v[7] << 16);
            *reinterpret_cast<uint4*>(ent) = q;
        } else {
#pragma unroll
            for (int b = 0; b < XSUB; ++b) ent[b] = v[b];
        }
    }
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

// Sub-bin of x counted from the chunk's first source cell, clamped to
// [lo, hi]: the FP32 expression of k_stabilise, so it is monotone in x and
// agrees with the sub-bins the table was built from.
__device__ __forceinline__ int sub_bin(float x, float xlo, float invs, int base, int lo, int hi)
{
    const int b = __float2int_rd(__fmul_rn(__fsub_rn(x, xlo), invs)) - base;
    return min(max(b, lo), hi);
}

// The 9 x-windows of one target: per row r, the sources whose sub-bin lies
// between those of x - w_r and x + w_r, w_r = sqrt(rc^2 - d_yz^2) (inflated
// by 2e-5 relative and the slack; negative d_yz^2 headroom = row out of
// reach, empty window), and inside the target's cells cx - 1 .. cx + 1 (the
// 27-cell stencil of the cell list, so a window never depends on how far
// the chunk extends).  Every source of the stencil that the pair test
// accepts is inside; the rest fail the test.  Windows are [j[r], je[r]) in
// the table's indices.
template <class E, int RB>
__device__ __forceinline__ void target_windows(const E (*tbl)[RB], uint32_t coarse_mask,
                                               const SysDesc& d, float xt, float yt, float zt, int cy,
                                               int cz, int base, int (&j)[9], int (&je)[9])
{
    const Faces f = faces_of(d, yt, zt, cy, cz);
    const float rcm2 = d.rc2 * 1.00002f;
    const float xlo = d.g.lo[0], slack = d.slack, invs = d.g.inv_w[0] * (float)XSUB;
    const int nx = d.g.n[0];
    const int cx = axis_cell(xt, xlo, d.g.inv_w[0], nx);
    const int lo = XSUB * max(cx - 1, 0) - base;
    const int hi = XSUB * (min(cx + 1, nx - 1) + 1) - base - 1;
#pragma unroll
    for (int rr = 0; rr < 9; ++rr) {
        const int dy = rr % 3 - 1, dz = rr / 3 - 1;
        const float ey = dy < 0 ? f.y_lo : (dy > 0 ? f.y_hi : 0.f);
        const float ez = dz < 0 ? f.z_lo : (dz > 0 ? f.z_hi : 0.f);
        const float t = rcm2 - fmaf(ey, ey, ez * ez);
        const float tt = fmaxf(t, 1e-30f);
        const float w = tt * rsqrtf(tt) + slack;
        const int b0 = sub_bin(xt - w, xlo, invs, base, lo, hi);
        int b1 = sub_bin(xt + w, xlo, invs, base, lo, hi) + 1;
        if ((coarse_mask >> rr) & 1u) b1 = (b1 + XSUB - 1) / XSUB * XSUB;
        const int first = (int)tbl[rr][b0];
        j[rr] = first;
        je[rr] = t > 0.f ? (int)tbl[rr][b1] : first;
    }
}

// 1.0f if a < b and u != v, else 0.0f (PTX set with a float destination):
// the pair test with the self pair excluded by identity (u, v the stable
// slots of source and target).
__device__ __forceinline__ float lt_ne_mask(float a, float b, float u, float v)
{
    float m;
    asm("{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %3, %4;\n\t"
        "set.lt.and.f32.f32 %0, %1, %2, p;\n\t}"
        : "=f"(m) : "f"(a), "f"(b), "r"(__float_as_uint(u)), "r"(__float_as_uint(v)));
    return m;
}

// Two targets a and b against one candidate source with packed FP32
// (f32x2) arithmetic: element .x belongs to target a, .y to target b, and
// every element is rounded exactly as the scalar steps of Sums::pair_nb
// round it, candidate after candidate, so each target's sums are those of
// the sequential scalar loop.  The pair test gives a 1/0 mask m and the
// term is K = value * m, so a candidate that fails it (the other target's,
// a row's sentinel slots, the target itself) contributes an exact zero,
// which leaves the plain sums as they were.  The compensated sums take the same zero through the mask: with
// y = t - c*m, u = v + y, c' = (u - v) - y and c <- c*(1 - m) + c', a
// rejected candidate leaves v and c unchanged (up to the sign of a zero c)
// and an accepted one is the Kahan step exactly.  Compensations are kept
// negated (cn = -c) so that every step is one add or fma.
// gauss_fine for two targets with packed FP32 arithmetic (each element
// rounded as the scalar steps round it).
__device__ __forceinline__ float2 neg2(float2 v) { return make_float2(-v.x, -v.y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e)
{
    s = __fadd2_rn(a, b);
    const float2 bb = sub2(s, a);
    e = __fadd2_rn(sub2(a, sub2(s, bb)), sub2(b, bb));
}
__device__ __forceinline__ float2 gauss_fine2(float2 dx, float2 dy, float2 dz, float2 th, float2 tl)
{
    const float2 px = __fmul2_rn(dx, dx), ex = __ffma2_rn(dx, dx, neg2(px));
    const float2 py = __fmul2_rn(dy, dy), ey = __ffma2_rn(dy, dy, neg2(py));
    const float2 pz = __fmul2_rn(dz, dz), ez = __ffma2_rn(dz, dz, neg2(pz));
    float2 s1, e1, s2, e2;
    two_sum2(px, py, s1, e1);
    two_sum2(s1, pz, s2, e2);
    const float2 uh = __fmul2_rn(s2, th);
    const float2 ue = __ffma2_rn(s2, th, neg2(uh));
    const float2 es = __fadd2_rn(__fadd2_rn(ex, ey), __fadd2_rn(ez, __fadd2_rn(e1, e2)));
    float2 c = __ffma2_rn(th, es, __ffma2_rn(tl, s2, ue));
    c = make_float2(fminf(fmaxf(c.x, -1.f), 1.f), fminf(fmaxf(c.y, -1.f), 1.f));
    const float2 k0 = make_float2(ex2_approx(uh.x), ex2_approx(uh.y));
    return __ffma2_rn(__fmul2_rn(k0, c), make_float2(LN2_F, LN2_F), k0);
}

template <class Acc, int KERNEL>
struct PairSumsT {
    static constexpr bool kahan = std::is_same<Acc, KahanAcc>::value;
    float2 s = make_float2(0.f, 0.f), vx = make_float2(0.f, 0.f), vy = make_float2(0.f, 0.f),
           vz = make_float2(0.f, 0.f), n = make_float2(0.f, 0.f);
    float2 cs = make_float2(0.f, 0.f), cx = make_float2(0.f, 0.f), cy = make_float2(0.f, 0.f),
           cz = make_float2(0.f, 0.f);

    __device__ __forceinline__ static void comp_add(float2& v, float2& cn, float2 t, float2 m, float2 nm)
    {
        const float2 m1 = make_float2(-1.f, -1.f);
        const float2 y = __ffma2_rn(cn, m, t);      // t - c (t when rejected)
        const float2 u = __fadd2_rn(v, y);
        const float2 d = __ffma2_rn(v, m1, u);      // u - v
        const float2 cn1 = __ffma2_rn(d, m1, y);    // -((u - v) - y)
        cn = __ffma2_rn(cn, nm, cn1);
        v = u;
    }

    __device__ __forceinline__ void cand(const float4& p, const float4& ta, const float4& tb, float rc2,
                                         float2 ks, const KParams& kp)
    {
        // offsets as packed adds of the negated targets to the source
        // coordinate in both halves: p - t rounded exactly as the scalar
        // subtraction (the negation is exact), in three packed adds instead
        // of six scalar ones (measured 2.5 % faster than the scalar form)
        const float2 dx = __fadd2_rn(make_float2(p.x, p.x), make_float2(-ta.x, -tb.x));
        const float2 dy = __fadd2_rn(make_float2(p.y, p.y), make_float2(-ta.y, -tb.y));
        const float2 dz = __fadd2_rn(make_float2(p.z, p.z), make_float2(-ta.z, -tb.z));
        const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
        const float2 m = make_float2(lt_ne_mask(r2.x, rc2, p.w, ta.w), lt_ne_mask(r2.y, rc2, p.w, tb.w));
        float2 K;
        if constexpr (KERNEL == KERNEL_GAUSSIAN) {
            const float2 t = __fmul2_rn(r2, ks);
            K = __fmul2_rn(make_float2(ex2_approx(t.x), ex2_approx(t.y)), m);
        } else if constexpr (KERNEL == KERNEL_GAUSSIAN_FINE) {
            K = __fmul2_rn(gauss_fine2(dx, dy, dz, ks, make_float2(kp.tl, kp.tl)), m);
        } else if constexpr (KERNEL == KERNEL_LOWFLOP) {
            K = m;
        } else {
            // kernel_value's Lennard-Jones steps, element by element
            const float2 rs2 = __ffma2_rn(make_float2(0.01f, 0.01f), ks, r2);
            const float2 sr = __fmul2_rn(ks, make_float2(__frcp_rn(rs2.x), __frcp_rn(rs2.y)));
            const float2 s3 = __fmul2_rn(__fmul2_rn(sr, sr), sr);
            const float2 q = __ffma2_rn(s3, make_float2(-1.f, -1.f), __fmul2_rn(s3, s3));
            float2 e = __fmul2_rn(make_float2(4.0f, 4.0f), q);
            if constexpr (KERNEL == KERNEL_HIGHFLOP) {
                const float2 one = make_float2(kp.one, kp.one), zero = make_float2(kp.zero, kp.zero);
#pragma unroll
                for (int i = 0; i < 75; ++i) e = __ffma2_rn(e, one, zero);
            }
            K = __fmul2_rn(e, m);
        }
        if constexpr (!kahan) {
            s = __fadd2_rn(s, K);
            vx = __ffma2_rn(dx, K, vx);
            vy = __ffma2_rn(dy, K, vy);
            vz = __ffma2_rn(dz, K, vz);
        } else {
            const float2 nm = __ffma2_rn(m, make_float2(-1.f, -1.f), make_float2(1.f, 1.f));
            comp_add(s, cs, K, m, nm);
            comp_add(vx, cx, __fmul2_rn(dx, K), m, nm);
            comp_add(vy, cy, __fmul2_rn(dy, K), m, nm);
            comp_add(vz, cz, __fmul2_rn(dz, K), m, nm);
        }
        n = __fadd2_rn(n, m);
    }

    // target a's (second = false) or b's sums into r
    __device__ __forceinline__ void to(Sums<Acc, KERNEL>& r, bool second) const
    {
        r.s.v = second ? s.y : s.x;
        r.vx.v = second ? vx.y : vx.x;
        r.vy.v = second ? vy.y : vy.x;
        r.vz.v = second ? vz.y : vz.x;
        r.n = (uint32_t)(second ? n.y : n.x);  // exact: at most 2^24 neighbours
    }
};

using PairSums = PairSumsT<PlainAcc, KERNEL_GAUSSIAN>;

template <class Acc, int KERNEL>
__host__ __device__ constexpr bool packed_path()
{
    return std::is_same<Acc, PlainAcc>::value && KERNEL == KERNEL_GAUSSIAN;
}

// The candidates [j, je) of one window for one target, in order, one at a
// time (every path that does not pack two targets).
template <class Acc, int KERNEL>
__device__ __forceinline__ void window_sums(const float4* src, int j, int je, float xt, float yt,
                                            float zt, uint32_t slot, float rc2, const KParams& kp,
                                            Sums<Acc, KERNEL>& r)
{
    for (; j < je; ++j) {
        const float4 s0 = src[j];
        r.pair_nb(__fsub_rn(s0.x, xt), __fsub_rn(s0.y, yt), __fsub_rn(s0.z, zt), rc2, kp,
                  __float_as_uint(s0.w) == slot);
    }
}

// Mode 0, two targets a and b of one thread (b may repeat a when the thread
// has one target): per row the union of their windows goes to the thread's
// column of `win` (rows where both are empty dropped), then all of them are
// walked in one loop, so that a lane whose window in one row is short goes
// on with the next row instead of idling until the warp's longest window of
// that row ends.  Every source read is evaluated against both targets: one
// shared-memory load feeds two pair evaluations.  Each target's terms come
// in the order of its own windows (row by row, x-sorted), as in the
// per-target loops of the other paths, so every path gives the same sums.
template <int CAP, int RB, int WT>
__device__ __forceinline__ void target_pair_sums_staged(const float4* buf, const uint16_t (*tbl)[RB],
                                                        uint32_t coarse_mask, const SysDesc& d,
                                                        uint32_t (*win)[WT], unsigned tid,
                                                        const float4& ta, const float4& tb, int cy,
                                                        int cz, int base, const KParams& kp,
                                                        Sums<PlainAcc, KERNEL_GAUSSIAN>& ra,
                                                        Sums<PlainAcc, KERNEL_GAUSSIAN>& rb, Ctrl* ctrl)
{
    int nw = 0;
    {
        int ja[9], jea[9], jb[9], jeb[9];
        target_windows(tbl, coarse_mask, d, ta.x, ta.y, ta.z, cy, cz, base, ja, jea);
        target_windows(tbl, coarse_mask, d, tb.x, tb.y, tb.z, cy, cz, base, jb, jeb);
#pragma unroll
        for (int rr = 0; rr < 9; ++rr) {
            const bool ea = jea[rr] > ja[rr], eb = jeb[rr] > jb[rr];
            const int lo = ea ? (eb ? min(ja[rr], jb[rr]) : ja[rr]) : jb[rr];
            const int hi = ea ? (eb ? max(jea[rr], jeb[rr]) : jea[rr]) : jeb[rr];
            if (ea || eb) win[nw++][tid] = (uint32_t)lo * 16u | ((uint32_t)hi * 16u << 16);
        }
    }
    // nw >= 1: the window of a's own row holds a
#ifdef PI_CHECK
    if (!PI_BOUNDS(ctrl, nw > 0 ? 0 : 1, 1, CS_STAGED_BUF)) return;
#endif
    const float rc2 = d.rc2;
    const float2 ks = make_float2(kp.t, kp.t);
    PairSums ps;
    // shared-window addresses: candidates, this thread's window words
    const uint32_t cb = smem_addr(buf), wb = smem_addr(&win[0][tid]);
    constexpr uint32_t WSTEP = (uint32_t)WT * 4u;
    const uint32_t we = wb + (uint32_t)nw * WSTEP;
    uint32_t wa = wb;
    const uint32_t w0 = lds_u32(wa);
    uint32_t c = cb + (w0 & 0xffffu), ce = cb + (w0 >> 16);
    // All windows in one loop with the switch written as selects, so no lane
    // waits for the others at the end of a window (a lane leaves after its
    // last one).  Four sources per trip; the up to three slots read past a
    // window's end (the same row outside the windows, or the row's sentinel
    // slots) add exact zeros.
    do {
        if (!PI_BOUNDS(ctrl, (uint64_t)((c - cb) / 16u) + 3u, CAP + 1, CS_STAGED_BUF)) break;
        const float4 s0 = lds_f4(c), s1 = lds_f4(c + 16u), s2 = lds_f4(c + 32u), s3 = lds_f4(c + 48u);
        ps.cand(s0, ta, tb, rc2, ks, kp);
        ps.cand(s1, ta, tb, rc2, ks, kp);
        ps.cand(s2, ta, tb, rc2, ks, kp);
        ps.cand(s3, ta, tb, rc2, ks, kp);
        c += 64u;
        const bool sw = c >= ce;
        wa += sw ? WSTEP : 0u;
        const uint32_t wn = lds_u32(wa);
        c = sw ? cb + (wn & 0xffffu) : c;
        ce = sw ? cb + (wn >> 16) : ce;
    } while (wa < we);
    ps.to(ra, false);
    ps.to(rb, true);
}

// Mode 0, one target, one candidate at a time over its own windows (the
// kernels and precision modes without the packed two-target path).
template <int RB, class Acc, int KERNEL>
__device__ __forceinline__ void target_sums_staged(const float4* buf, const uint16_t (*tbl)[RB],
                                                   uint32_t coarse_mask, const SysDesc& d, const float4& t,
                                                   int cy, int cz, int base, const KParams& kp,
                                                   Sums<Acc, KERNEL>& r)
{
    int j[9], je[9];
    target_windows(tbl, coarse_mask, d, t.x, t.y, t.z, cy, cz, base, j, je);
    const uint32_t slot = __float_as_uint(t.w);
#pragma unroll 1
    for (int rr = 0; rr < 9; ++rr)
        window_sums<Acc, KERNEL>(buf, j[rr], je[rr], t.x, t.y, t.z, slot, d.rc2, kp, r);
}

// Mode 1, one target: the same windows, read from P in global memory.
template <class Acc, int KERNEL>
__device__ __forceinline__ void target_sums_global(const float4* P, const uint32_t (*tbl)[RB_GLOBAL],
                                                   uint32_t coarse_mask, const SysDesc& d, const float4& t,
                                                   int cy, int cz, int base, const KParams& kp,
                                                   Sums<Acc, KERNEL>& r)
{
    int j[9], je[9];
    target_windows(tbl, coarse_mask, d, t.x, t.y, t.z, cy, cz, base, j, je);
    const uint32_t slot = __float_as_uint(t.w);
#pragma unroll 1
    for (int rr = 0; rr < 9; ++rr)
        window_sums<Acc, KERNEL>(P, j[rr], je[rr], t.x, t.y, t.z, slot, d.rc2, kp, r);
}

// The sums of a thread's targets qa and qb = qa + 1 of a chunk (qb only if
// has_b), whichever path the chunk and the kernel take, stored.  `first`
// gives a target's position: staged index in mode 0, P index in mode 1.
template <int CAP, int RB, int WT, class Acc, int KERNEL>
__device__ __forceinline__ void chunk_pair(const InteractArgs& a, const float4* buf,
                                           const uint16_t (*tbl_s)[RB], const uint32_t (*tbl_g)[RB_GLOBAL],
                                           uint32_t coarse_mask, const SysDesc& d, uint32_t (*win)[WT],
                                           unsigned tid, int mode, int first, int qa, bool has_b, int cy,
                                           int cz, int base, const KParams& kp)
{
    const int qb = has_b ? qa + 1 : qa;
    const float4 ta = mode == 0 ? buf[first + qa] : a.P[first + qa];
    const float4 tb = mode == 0 ? buf[first + qb] : a.P[first + qb];
    Sums<Acc, KERNEL> ra, rb;
    if (mode == 0) {
        if constexpr (packed_path<Acc, KERNEL>()) {
            target_pair_sums_staged<CAP, RB, WT>(buf, tbl_s, coarse_mask, d, win, tid, ta, tb, cy, cz, base, kp,
                                                 ra, rb, a.ctrl);
        } else {
            target_sums_staged<RB, Acc, KERNEL>(buf, tbl_s, coarse_mask, d, ta, cy, cz, base, kp, ra);
            if (has_b) target_sums_staged<RB, Acc, KERNEL>(buf, tbl_s, coarse_mask, d, tb, cy, cz, base, kp, rb);
        }
    } else {
        target_sums_global<Acc, KERNEL>(a.P, tbl_g, coarse_mask, d, ta, cy, cz, base, kp, ra);
        if (has_b) target_sums_global<Acc, KERNEL>(a.P, tbl_g, coarse_mask, d, tb, cy, cz, base, kp, rb);
    }
    store_out(a, __float_as_uint(ta.w), ra);
    if (has_b) store_out(a, __float_as_uint(tb.w), rb);
}

template <class T, class Acc, int KERNEL>
__global__ void __launch_bounds__(T::NT, T::MINB) k_interact_tiled(InteractArgs a)
{
    constexpr int NT = T::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<T>& sm = *reinterpret_cast<Smem<T>*>(smem_raw);

    pdl_trigger();
    pdl_wait();
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctrl->work[(a.seq + 1u) & 1u] = 0u;
    const unsigned tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    if (tid == 0) {
        // the error word once per CTA (see cta_ctrl_words)
        sm.failed = load_error(a.ctrl) != 0u;
        sm.buf[T::CAP] = sentinel();
        bar_init(&sm.bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (sm.failed) return;
    uint32_t phase = 0;

    for (;;) {
        if (tid == 0) {
            const uint32_t item = atomicAdd(&a.ctrl->work[a.seq & 1u], 1u);
            sm.has_row = item < a.work;
            if (item < a.work) {
                const int sid = a.sy.S == 1 ? 0 : find_system(a.sy.wbase, a.sy.S, item);
                sm.d = a.sy.sys[sid];
                sm.kp = kparams(a, sid);
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
        const int cy = (int)(row % (uint32_t)ny), cz = (int)(row / (uint32_t)ny);
        const uint32_t rb0 = d.cell_base + (uint32_t)nx * row;

        const int xe = sm.xe;
        for (int x0 = sm.xs; x0 < xe;) {
            if (warp == 0) {
                if (lane == 0) sm.coarse_mask = 0u;
                plan_chunk<T>(a, d, sm.plan, x0, xe, cy, cz, lane);
                __syncwarp();
                if (sm.plan.mode == 0) write_row_pads<T::CAP>(sm.buf, sm.plan, lane, a.ctrl);
                if (lane == 0 && sm.plan.mode == 0 && rows_fit<T::CAP>(sm.plan, a.ctrl)) {
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
            const int x1 = p.x1, mode = p.mode;
            const int ncell = p.xb - p.xa + 1;
            // lookup tables, built while the bulk copies are in flight
            if (mode == 0)
                build_table<NT>(a, d, p, cy, cz, ncell, sm.tbl.staged, &sm.coarse_mask, tid);
            else
                build_table<NT>(a, d, p, cy, cz, ncell, sm.tbl.global, &sm.coarse_mask, tid);
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
            const uint32_t tb0 = a.offsets[rb0 + x0], te = a.offsets[rb0 + x1];
            const int ntarget = (int)(te - tb0);
            const uint32_t tb = tb0 + ROW_PADS * (d.row_base + row);  // P index of the first target
            // staged index of the first target (the centre row is row 4)
            const int t0 = p.sbeg[4] + (int)(tb - p.gbeg[4]);
            const int base = XSUB * p.xa;
            if (!sm.failed) {
                const KParams kp = sm.kp;
                const int first = mode == 0 ? t0 : (int)tb;
                for (int q0 = 0; q0 < ntarget; q0 += 2 * NT) {
                    const int qa = q0 + 2 * (int)tid;
                    if (qa >= ntarget) continue;
                    chunk_pair<T::CAP, T::RB, NT, Acc, KERNEL>(a, sm.buf, sm.tbl.staged, sm.tbl.global,
                                                               sm.coarse_mask, sm.d, sm.win, tid, mode, first,
                                                               qa, qa + 1 < ntarget, cy, cz, base, kp);
                }
            }
            __syncthreads();
            x0 = x1;
        }
    }
}

// ---- warp-specialised tiled interaction -----------------------------------------
//
// The same chunks, windows and per-target sums as k_interact_tiled, but the
// chunk set-up no longer stalls the CTA: one producer warp plans a chunk,
// issues its bulk copies and builds its lookup table into one of NS stage
// buffers while W consumer warps work on the chunks already staged.  The
// consumers take 32-target groups of a chunk from a counter, so a warp that
// is done with its groups goes on with the next chunk instead of waiting for
// the slowest warp.  Hand-over is by mbarriers: `full` (the producer's 32
// lanes arrive after writing the stage, plus the bytes of the bulk copies)
// and `empty` (every consumer lane arrives when its warp has left the
// chunk).  Every wait is bounded.

template <int W_, int CAP_, int NS_, int MAXLX_, int MINB_, int GMAX_>
struct WsTile {
    static constexpr int W = W_;              // consumer warps
    static constexpr int CAP = CAP_;          // staged particles per stage
    static constexpr int NS = NS_;            // stages
    static constexpr int MAXLX = MAXLX_;      // target cells per chunk along X
    static constexpr int MINB = MINB_;        // CTAs per SM the budget is sized for
    static constexpr int TT = 64 * GMAX_;     // most targets per chunk (planner limit)
    static constexpr int THREADS = 32 * (W + 1);
    static constexpr int RB = ((MAXLX + 2) * XSUB + 1 + 7) / 8 * 8;
};
using Ws4 = WsTile<4, 2432, 2, SEG_CELLS, 2, 4>;
using Ws8 = WsTile<8, 2432, 2, SEG_CELLS, 2, 4>;

template <class T>
struct WsStage {
    float4 buf[T::CAP + 1];  // staged rows; buf[CAP] is the sentinel
    union {
        __align__(16) uint16_t staged[9][T::RB];
        uint32_t global[9][RB_GLOBAL];
    } tbl;
    Plan plan;
    SysDesc d;
    float t;               // kernel scale of the chunk's system
    uint32_t coarse_mask;  // bit r: row r holds a cell without sub-bin starts
    int cy, cz;            // the chunk's X-row
    uint32_t tb;           // P index of its first target
    int ntarget, ngroups;
    int next_group;        // next 64-target group (two per lane) handed to a consumer warp
    int done;              // set instead of a chunk when the work is over
    uint64_t full, empty;
};

template <class T>
struct WsSmem {
    WsStage<T> st[T::NS];
    uint32_t win[10][32 * T::W];  // per consumer thread: its windows (see target_pair_sums_staged)
    int failed;
};

template <class T>
constexpr bool ws_fits_sm()
{
    return T::MINB * (sizeof(WsSmem<T>) + 1024) <= 228u * 1024u;
}
static_assert(ws_fits_sm<Ws4>() && ws_fits_sm<Ws8>(),
              "warp-specialised shapes exceed the shared memory of their CTAs per SM");

__device__ __forceinline__ void bar_expect_tx_only(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Bounded wait of a whole warp; the outcome is the same on every lane (a
// lane whose wait ran out makes the warp give up), so that the warp stays
// converged for the shuffles that follow.
template <class T>
__device__ __forceinline__ bool ws_wait(WsSmem<T>& sm, uint64_t* bar, uint32_t parity, uint64_t limit,
                                        Ctrl* ctrl)
{
    const bool got = bar_wait_bounded(bar, parity, limit);
    if (__all_sync(0xffffffffu, got)) return true;
    if ((threadIdx.x & 31u) == 0) {
        *((volatile int*)&sm.failed) = 1;
        atomicOr(&ctrl->error, ERR_TIMEOUT);
    }
    return false;
}

template <class T>
__device__ void ws_producer(const InteractArgs& a, WsSmem<T>& sm, unsigned lane)
{
    constexpr int NS = T::NS;
    // per stage: its last use handed over, and whether that use had bulk
    // copies (those of earlier uses have landed: the consumers waited for
    // them before releasing the stage)
    int last_use[NS];
    bool copies[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        last_use[s] = -1;
        copies[s] = false;
    }
    uint32_t v = 0;  // chunks handed over so far
    bool ok = true;
    while (ok) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(&a.ctrl->work[a.seq & 1u], 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= a.work) break;
        const int sid = a.sy.S == 1 ? 0 : find_system(a.sy.wbase, a.sy.S, item);
        const SysDesc d = a.sy.sys[sid];
        const float t = a.kscale ? a.kscale[sid] : a.kscale0;
        const uint32_t local = item - d.work_base;
        const uint32_t seg = local % d.nseg, row = local / d.nseg;
        const int nx = d.g.n[0], ny = d.g.n[1];
        const int cy = (int)(row % (uint32_t)ny), cz = (int)(row / (uint32_t)ny);
        const uint32_t rb0 = d.cell_base + (uint32_t)nx * row;
        const int xs = (int)seg * SEG_CELLS, xe = min(nx, (int)(seg + 1) * SEG_CELLS);
        for (int x0 = xs; x0 < xe;) {
            const int s = (int)(v % NS);
            const uint32_t u = v / NS;
            WsStage<T>& st = sm.st[s];
            if (u > 0 && !ws_wait(sm, &st.empty, (u - 1u) & 1u, a.wait_limit_ns, a.ctrl)) {
                ok = false;
                break;
            }
            if (lane == 0) st.coarse_mask = 0u;
            __syncwarp();
            plan_chunk<T>(a, d, st.plan, x0, xe, cy, cz, lane);
            __syncwarp();
            const Plan& p = st.plan;
            const int x1 = p.x1, mode = p.mode, ncell = p.xb - p.xa + 1;
            if (mode == 0) write_row_pads<T::CAP>(st.buf, p, lane, a.ctrl);
            if (lane == 0 && mode == 0 && rows_fit<T::CAP>(p, a.ctrl)) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                bar_expect_tx_only(&st.full, (uint32_t)p.total * 16u);
                for (int rr = 0; rr < 9; ++rr)
                    if (p.rlen[rr] > 0)
                        bulk_g2s(&st.buf[p.sbeg[rr]], a.P + p.gbeg[rr], (uint32_t)p.rlen[rr] * 16u, &st.full);
            }
            last_use[s] = (int)u;
            copies[s] = mode == 0;
            if (mode == 0) {
                build_table<32>(a, d, p, cy, cz, ncell, st.tbl.staged, &st.coarse_mask, lane);
            } else {
                build_table<32>(a, d, p, cy, cz, ncell, st.tbl.global, &st.coarse_mask, lane);
            }
            if (lane == 0) {
                const uint32_t tb0 = a.offsets[rb0 + x0];
                const int nt = (int)(a.offsets[rb0 + x1] - tb0);
                const uint32_t tb = tb0 + ROW_PADS * (d.row_base + row);  // P index
                st.d = d;
                st.t = t;
                st.cy = cy;
                st.cz = cz;
                st.tb = tb;
                st.ntarget = nt;
                st.ngroups = (nt + 63) / 64;
                st.next_group = 0;
                st.done = 0;
            }
            bar_arrive(&st.full);  // every lane: its table entries are written
            ++v;
            x0 = x1;
        }
    }
    if (ok) {
        const int s = (int)(v % NS);
        const uint32_t u = v / NS;
        WsStage<T>& st = sm.st[s];
        if (u == 0 || ws_wait(sm, &st.empty, (u - 1u) & 1u, a.wait_limit_ns, a.ctrl)) {
            if (lane == 0) st.done = 1;
            bar_arrive(&st.full);
            return;  // the consumers wait for every handed-over stage before they leave
        }
    }
    // after a failure, let this CTA's bulk copies in flight land first
#pragma unroll
    for (int s = 0; s < NS; ++s)
        if (copies[s]) bar_wait_bounded(&sm.st[s].full, (uint32_t)last_use[s] & 1u, a.wait_limit_ns);
}

template <class T, class Acc, int KERNEL>
__device__ void ws_consumer(const InteractArgs& a, WsSmem<T>& sm, unsigned tid, unsigned lane)
{
    constexpr int NS = T::NS;
    for (uint32_t v = 0;; ++v) {
        const int s = (int)(v % NS);
        const uint32_t u = v / NS;
        WsStage<T>& st = sm.st[s];
        if (!ws_wait(sm, &st.full, u & 1u, a.wait_limit_ns, a.ctrl)) return;
        if (st.done) return;
        const Plan& p = st.plan;
        const int mode = p.mode, base = XSUB * p.xa, cy = st.cy, cz = st.cz, nt = st.ntarget,
                  ng = st.ngroups;
        const uint32_t tb = st.tb;
        const int first = mode == 0 ? p.sbeg[4] + (int)(tb - p.gbeg[4]) : (int)tb;
        const KParams kp{st.t, 0.f, a.one, a.zero};  // the fine Gaussian never runs here
        for (;;) {
            int g = 0;
            if (lane == 0) g = atomicAdd(&st.next_group, 1);
            g = __shfl_sync(0xffffffffu, g, 0);
            if (g >= ng) break;
            const int qa = 64 * g + 2 * (int)lane;
            if (qa < nt)
                chunk_pair<T::CAP, T::RB, 32 * T::W, Acc, KERNEL>(a, st.buf, st.tbl.staged, st.tbl.global,
                                                                  st.coarse_mask, st.d, sm.win, tid, mode,
                                                                  first, qa, qa + 1 < nt, cy, cz, base, kp);
        }
        __syncwarp();
        bar_arrive(&st.empty);
        if (__any_sync(0xffffffffu, *((volatile int*)&sm.failed) != 0)) return;
    }
}

template <class T, class Acc, int KERNEL>
__global__ void __launch_bounds__(T::THREADS, T::MINB) k_interact_ws(InteractArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WsSmem<T>& sm = *reinterpret_cast<WsSmem<T>*>(smem_raw);
    const unsigned tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    pdl_trigger();
    pdl_wait();
    if (tid == 0) {
        if (blockIdx.x == 0) a.ctrl->work[(a.seq + 1u) & 1u] = 0u;
        sm.failed = load_error(a.ctrl) != 0u;
        for (int s = 0; s < T::NS; ++s) {
            sm.st[s].buf[T::CAP] = sentinel();
            bar_init(&sm.st[s].full, 32);
            bar_init(&sm.st[s].empty, 32 * T::W);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (sm.failed) return;
    if (warp == (unsigned)T::W)
        ws_producer<T>(a, sm, lane);
    else
        ws_consumer<T, Acc, KERNEL>(a, sm, tid, lane);
}

// ---- direct interaction (no staging) ------------------------------------------
//
// The same windows, pairs of targets and summation order as the tiled
// kernels, without shared-memory staging: one thread takes two consecutive
// targets of the sorted order, reads the sub-bin starts of its windows from
// the offsets and `xbins` in global memory, and loads every source straight
// from P through L1 (neighbouring threads work on the same rows, so the
// loads hit).  No chunks, no barriers: only the window lists live in shared
// memory, so occupancy is set by registers alone.

constexpr int DIRECT_THREADS = DIRECT_BLOCK;

// First index in [lo, hi) of P whose x is >= v (strict: > v); hi if none.
__device__ __noinline__ uint32_t x_bound(const float4* P, uint32_t lo, uint32_t hi, float v, bool strict)
{
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        const float xm = __ldg(&P[mid].x);
        const bool left = strict ? !(xm > v) : (xm < v);
        lo = left ? mid + 1u : lo;
        hi = left ? hi : mid;
    }
    return lo;
}

// First index of P whose sub-bin in the row starting at cell `rb` is >= b
// (b counted from the row's first cell); `upper`: round a sub-bin of a cell
// without sub-bin starts up to the cell's end instead of down to its start.
// `dense` is set when the lookup read the sub-bin word of a cell with more
// than DENSE_CELL members (left unchanged otherwise).
__device__ __forceinline__ uint32_t sub_bin_start(const InteractArgs& a, uint32_t rb, int b, bool upper,
                                                  bool& dense)
{
    const uint32_t k = (uint32_t)(b >> 3), sub = (uint32_t)(b & 7);
#ifdef PI_CHECK
    // offsets has C + 1 entries, xbins C: the start of a cell may be read
    // at index C (the end of the last row), a sub-bin word only inside
    const uint64_t c_all = __ldg(a.sy.cbase + a.sy.S);
    if (!PI_BOUNDS(a.ctrl, (uint64_t)rb + k, c_all + 1u, CS_DIRECT_LOOKUP)) return 0u;
    if (sub != 0 && !PI_BOUNDS(a.ctrl, (uint64_t)rb + k, c_all, CS_DIRECT_LOOKUP)) return 0u;
#endif
    const uint32_t start = __ldg(a.offsets + rb + k);
    if (sub == 0) return start;
    const uint2 w = __ldg(a.xbins + rb + k);
    dense = (w.y >> 24) != 0u;
    if ((w.y >> 24) & XBIN_COARSE) return upper ? __ldg(a.offsets + rb + k + 1) : start;
    const uint32_t word = sub <= 4 ? w.x : w.y;
    return start + ((word >> (8 * ((sub - 1) & 3))) & 255u);
}

// The x-windows of a group of G targets of one X-row (see target_windows;
// here the lookups read global memory), one range [ulo, uhi) of P indices
// per neighbour row, left unchanged for a row where the range is empty.
// The union is taken in x before the lookups: the smallest x - w_r and the
// largest x + w_r over the targets that have the row, clamped to the cells
// next to the group's, give one sub-bin range and two lookups per row
// instead of two per target.  Sub-bins and their starts are monotone in x,
// so the range holds every target's own window; what else it may hold (the
// sub-bins between two disjoint windows) is outside every target's cutoff
// and adds exact zeros.
template <bool DENSE, int G>
__device__ __forceinline__ void group_windows_direct(const InteractArgs& a, const SysDesc& d, const float4 (&t)[G],
                                                     const int (&cx)[G], int cy, int cz, uint32_t (&ulo)[9],
                                                     uint32_t (&uhi)[9])
{
    Faces f[G];
    int cmin = cx[0], cmax = cx[0];
#pragma unroll
    for (int k = 0; k < G; ++k) {
        f[k] = faces_of(d, t[k].y, t[k].z, cy, cz);
        cmin = min(cmin, cx[k]);
        cmax = max(cmax, cx[k]);
    }
    const float rcm2 = d.rc2 * 1.00002f;
    const float xlo = d.g.lo[0], slack = d.slack, invs = d.g.inv_w[0] * (float)XSUB;
    const int nx = d.g.n[0], ny = d.g.n[1], nz = d.g.n[2];
    const int lo = XSUB * max(cmin - 1, 0);
    const int hi = XSUB * (min(cmax + 1, nx - 1) + 1) - 1;
#pragma unroll
    for (int rr = 0; rr < 9; ++rr) {
        const int dy = rr % 3 - 1, dz = rr / 3 - 1;
        const int by = cy + dy, bz = cz + dz;
        if (by < 0 || by >= ny || bz < 0 || bz >= nz) continue;
        float xl = INFINITY, xu = -INFINITY;
#pragma unroll
        for (int k = 0; k < G; ++k) {
            const float ey = dy < 0 ? f[k].y_lo : (dy > 0 ? f[k].y_hi : 0.f);
            const float ez = dz < 0 ? f[k].z_lo : (dz > 0 ? f[k].z_hi : 0.f);
            const float tw = rcm2 - fmaf(ey, ey, ez * ez);
            const float tt = fmaxf(tw, 1e-30f);
            const float w = tt * rsqrtf(tt) + slack;
            xl = tw > 0.f ? fminf(xl, t[k].x - w) : xl;
            xu = tw > 0.f ? fmaxf(xu, t[k].x + w) : xu;
        }
        if (!(xl <= xu)) continue;  // no target of the group reaches the row
        const uint32_t row = (uint32_t)by + (uint32_t)ny * (uint32_t)bz;
        const uint32_t rb = d.cell_base + (uint32_t)nx * row, pad = ROW_PADS * (d.row_base + row);
        const int b0 = sub_bin(xl, xlo, invs, 0, lo, hi);
        const int b1 = sub_bin(xu, xlo, invs, 0, lo, hi) + 1;
        bool dl = false, du = false;
        uint32_t j = sub_bin_start(a, rb, b0, false, dl) + pad;
        uint32_t je = sub_bin_start(a, rb, b1, true, du) + pad;
        // a bound inside a dense cell (b0's, or b1's when b1 is not the
        // cell's first sub-bin): the exact bound from a binary search of the
        // cell's x-sorted members.  Every source within the cutoff stays in
        // the window, so the sums do not change; only fewer zeros are added.
        if (DENSE && dl) {
            const uint32_t k = (uint32_t)(b0 >> 3);
            j = x_bound(a.P, __ldg(a.offsets + rb + k) + pad, __ldg(a.offsets + rb + k + 1) + pad, xl, false);
        }
        if (DENSE && du) {
            const uint32_t k = (uint32_t)(b1 >> 3);
            je = x_bound(a.P, __ldg(a.offsets + rb + k) + pad, __ldg(a.offsets + rb + k + 1) + pad, xu, true);
        }
        if (je > j) {
            ulo[rr] = j;
            uhi[rr] = je;
        }
    }
}

// A group of G targets (a target may repeat the one before it)
// of one X-row of one system: per row the union of their windows goes to
// column `col` of `win` (rows where all are empty dropped), and one loop walks
// all of them with the window switch written as selects (a lane leaves after
// its last window without waiting for the others at the end of each row),
// four sources per trip, each source evaluated against every target of the
// group, two at a time with packed arithmetic.  Candidates outside a
// target's own windows -- the other targets', up to three past a window's end
// (the same row outside the windows, or the row's sentinel slots), and for
// four targets one before a window's start -- add exact zeros, so each
// target's sums are those of the sequential loop over its own windows.
// Returns the source slots each target is evaluated against (the windows
// rounded up to whole four-source trips) in the counting copy (COUNT), else 0.
template <int WT, int G, bool DENSE, class Acc, int KERNEL, bool COUNT = false>
__device__ __forceinline__ uint32_t direct_group(const InteractArgs& a, const SysDesc& d, uint32_t (*win)[WT],
                                                 unsigned col, const float4 (&t)[G], const int (&cx)[G], int cy,
                                                 int cz, const KParams& kp, Sums<Acc, KERNEL> (&r)[G])
{
    static_assert(G % 2 == 0, "targets go in packed pairs");
    constexpr bool WIDE = G >= 4;
    int nw = 0;
    uint32_t slots = 0;
    {
        uint32_t ulo[9], uhi[9];
#pragma unroll
        for (int rr = 0; rr < 9; ++rr) {
            ulo[rr] = 0xffffffffu;
            uhi[rr] = 0u;
        }
        group_windows_direct<DENSE, G>(a, d, t, cx, cy, cz, ulo, uhi);
#pragma unroll
        for (int rr = 0; rr < 9; ++rr)
            if (uhi[rr] > ulo[rr] && PI_BOUNDS(a.ctrl, 2 * nw + 1, 18, CS_DIRECT_WIN)) {
                // four targets: an even start, so that trips of four
                // sources start on 32-byte boundaries of P (its base is
                // 256-byte aligned) and load as two 32-byte vectors; the
                // slot before a window is outside every target's cutoff (or
                // a row's sentinel) and adds zeros.  (Measured: faster for
                // four targets, slower for two, whose extra slot per window
                // costs more than the wider loads save.)
                const uint32_t lo = WIDE ? ulo[rr] & ~1u : ulo[rr];
                win[2 * nw][col] = lo;
                win[2 * nw + 1][col] = uhi[rr];
                if constexpr (COUNT) slots += (uhi[rr] - lo + 3u) & ~3u;
                ++nw;
            }
    }
    // nw >= 1: the window of the first target's own row holds it
#ifdef PI_CHECK
    // (a debug build whose checks dropped every window has nothing to read)
    if (!PI_BOUNDS(a.ctrl, nw > 0 ? 0 : 1, 1, CS_DIRECT_WIN)) {
#pragma unroll
        for (int k = 0; k < G; ++k) r[k] = Sums<Acc, KERNEL>();
        return 0u;
    }
#endif
    const float rc2 = d.rc2;
    const float2 ks = make_float2(kp.t, kp.t);
    PairSumsT<Acc, KERNEL> ps[G / 2];
    // the window words of this column by shared-window address
    const uint32_t wb = smem_addr(&win[0][col]);
    constexpr uint32_t WSTEP = (uint32_t)WT * 8u;  // one window = two rows of win
    const uint32_t we = wb + (uint32_t)nw * WSTEP;
    uint32_t wa = wb;
    uint32_t c = lds_u32(wa), ce = lds_u32(wa + WT * 4u);
    do {
        if (!PI_BOUNDS(a.ctrl, (uint64_t)c + 3u, a.np, CS_DIRECT_SRC) ||
            !PI_BOUNDS(a.ctrl, WIDE ? c & 1u : 0u, 1u, CS_DIRECT_SRC))
            break;
        const float4* q = a.P + c;
        float4 s0, s1, s2, s3;
        if constexpr (WIDE) {
            ldg_pair(q, s0, s1);
            ldg_pair(q + 2, s2, s3);
        } else {
            s0 = __ldg(q);
            s1 = __ldg(q + 1);
            s2 = __ldg(q + 2);
            s3 = __ldg(q + 3);
        }
#pragma unroll
        for (int h = 0; h < G / 2; ++h) {
            ps[h].cand(s0, t[2 * h], t[2 * h + 1], rc2, ks, kp);
            ps[h].cand(s1, t[2 * h], t[2 * h + 1], rc2, ks, kp);
            ps[h].cand(s2, t[2 * h], t[2 * h + 1], rc2, ks, kp);
            ps[h].cand(s3, t[2 * h], t[2 * h + 1], rc2, ks, kp);
        }
        c += 4u;
        const bool sw = c >= ce;
        wa += sw ? WSTEP : 0u;
        const uint32_t cn = lds_u32(wa), cen = lds_u32(wa + WT * 4u);
        c = sw ? cn : c;
        ce = sw ? cen : ce;
    } while (wa < we);
#pragma unroll
    for (int k = 0; k < G; ++k) ps[k / 2].to(r[k], (k & 1) != 0);
    return slots;
}

// Adds a thread's counted evaluations to the control block (the counting
// copy of the direct kernels, PI_OPT_COUNT_EVALS: one atomic per thread).
template <bool COUNT>
__device__ __forceinline__ void add_evals(const InteractArgs& a, unsigned long long ev)
{
    if constexpr (COUNT) {
        if (ev) atomicAdd(&a.ctrl->evals, ev);
    }
}

// The first P slot k0 of this thread's group of `per` consecutive slots
// and the end of the slots the launch covers: all of P, or -- for a launch
// over a list of P ranges (one tile shape for some systems of a batch) --
// the range this block falls in (blocks are dealt out range by range).
__device__ __forceinline__ void group_slots(const InteractArgs& a, uint32_t per, uint32_t& k0, uint32_t& kend)
{
    const uint32_t g = blockIdx.x * DIRECT_THREADS + threadIdx.x;
    if (!a.ranges) {
        k0 = per * g;
        kend = a.np;
        return;
    }
    const int r = find_system(a.rblock, a.nranges, blockIdx.x);
    const uint2 rg = __ldg(a.ranges + r);
    k0 = rg.x + per * (g - __ldg(a.rblock + r) * DIRECT_THREADS);
    kend = rg.y;
}

// Slots ka and ka + 1 of P below kend (either may be a sentinel or past
// the end).
template <int WT, bool DENSE, class Acc, int KERNEL, bool COUNT = false>
__device__ __forceinline__ void direct_slot_pair(const InteractArgs& a, uint32_t (*win)[WT], unsigned col,
                                                 uint32_t ka, uint32_t kend)
{
    if (ka >= kend) return;
    constexpr uint32_t NONE = 0xffffffffu;
    float4 ta = __ldg(a.P + ka);
    float4 t1 = ka + 1u < kend ? __ldg(a.P + ka + 1u) : ta;
    bool has_a = __float_as_uint(ta.w) != NONE, has_b = ka + 1u < kend && __float_as_uint(t1.w) != NONE;
    if (!has_a) {
        if (!has_b) return;
        ta = t1;
        has_a = true;
        has_b = false;
    }
    // the system of a target: from its stable slot (= sorted index)
    const int sid = a.sy.S == 1 ? 0 : find_system(a.sy.pbase, a.sy.S, __float_as_uint(ta.w));
    const int sid1 = (a.sy.S == 1 || !has_b) ? sid : find_system(a.sy.pbase, a.sy.S, __float_as_uint(t1.w));
    const SysDesc& d = a.sy.sys[sid];
    const Grid& g = d.g;
    const int cxa = axis_cell(ta.x, g.lo[0], g.inv_w[0], g.n[0]);
    const int cy = axis_cell(ta.y, g.lo[1], g.inv_w[1], g.n[1]);
    const int cz = axis_cell(ta.z, g.lo[2], g.inv_w[2], g.n[2]);
    const int cxb = axis_cell(t1.x, g.lo[0], g.inv_w[0], g.n[0]);
    // the two targets share the union of their windows when they lie in one
    // X-row of one system; otherwise each runs alone (b repeating a)
    const bool together = has_b && sid1 == sid && axis_cell(t1.y, g.lo[1], g.inv_w[1], g.n[1]) == cy &&
                          axis_cell(t1.z, g.lo[2], g.inv_w[2], g.n[2]) == cz;
    const KParams kp = kparams(a, sid);
    {
        const float4 t[2] = {ta, together ? t1 : ta};
        const int cx[2] = {cxa, together ? cxb : cxa};
        Sums<Acc, KERNEL> r[2];
        const uint32_t slots = direct_group<WT, 2, DENSE, Acc, KERNEL, COUNT>(a, d, win, col, t, cx, cy, cz, kp, r);
        add_evals<COUNT>(a, (unsigned long long)slots * (together ? 2u : 1u));
        store_out(a, __float_as_uint(ta.w), r[0]);
        if (together) store_out(a, __float_as_uint(t1.w), r[1]);
    }
    if (has_b && !together) {
        const SysDesc& d1 = a.sy.sys[sid1];
        const Grid& g1 = d1.g;
        const KParams kp1 = kparams(a, sid1);
        const int cx1 = axis_cell(t1.x, g1.lo[0], g1.inv_w[0], g1.n[0]);
        const int cy1 = axis_cell(t1.y, g1.lo[1], g1.inv_w[1], g1.n[1]);
        const int cz1 = axis_cell(t1.z, g1.lo[2], g1.inv_w[2], g1.n[2]);
        const float4 t[2] = {t1, t1};
        const int cx[2] = {cx1, cx1};
        Sums<Acc, KERNEL> r[2];
        add_evals<COUNT>(a, direct_group<WT, 2, DENSE, Acc, KERNEL, COUNT>(a, d1, win, col, t, cx, cy1, cz1, kp1, r));
        store_out(a, __float_as_uint(t1.w), r[0]);
    }
}

// The slot pair with exact window bounds in dense cells, out of line so that
// the common path keeps its code and registers.
template <class Acc, int KERNEL, bool COUNT = false>
__device__ __noinline__ void direct_slot_pair_dense(const InteractArgs& a, uint32_t (*win)[DIRECT_THREADS],
                                                    unsigned col, uint32_t ka, uint32_t kend)
{
    direct_slot_pair<DIRECT_THREADS, true, Acc, KERNEL, COUNT>(a, win, col, ka, kend);
}

// Resident CTAs per SM the direct kernel's registers are capped for.  The
// kernel waits mostly on source loads, so more resident warps pay more than
// registers: the plain Gaussian and low-FLOP kernels run 6 % faster with 8
// CTAs (32 warps, 64 registers) than with the 6 their 79 registers would
// allow, Lennard-Jones 10 % faster with 6 (80 registers) than with 5; the
// compensated sums are no faster at 7.
template <class Acc, int KERNEL>
__host__ __device__ constexpr int direct_min_blocks()
{
    return (std::is_same<Acc, PlainAcc>::value && (KERNEL == KERNEL_GAUSSIAN || KERNEL == KERNEL_LOWFLOP)) ? 8 : 6;
}

// Targets of P slots 2p and 2p + 1 per thread.  COUNT: the copy that also
// counts its evaluations (PI_OPT_COUNT_EVALS).
template <class Acc, int KERNEL, bool COUNT = false>
__global__ void __launch_bounds__(DIRECT_THREADS, (direct_min_blocks<Acc, KERNEL>()))
    k_interact_direct(InteractArgs a)
{
    __shared__ uint32_t win[20][DIRECT_THREADS];  // 9 windows (lo, hi) + one spare read after the last
    pdl_trigger();
    pdl_wait();  // the binning (or the previous interaction) has completed
    // keep the work counters of the tiled launches in step (see k_interact_tiled)
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctrl->work[(a.seq + 1u) & 1u] = 0u;
    // both control words in flight together, per thread (a per-CTA read
    // and barrier, cta_ctrl_words, measured 1 % slower here: the
    // evaluation hides these reads)
    const uint32_t err = load_error(a.ctrl);
    const uint32_t mpc = *((volatile const uint32_t*)&a.ctrl->max_per_cell);
    if (err) return;
    // grids with dense cells take the exact window bounds in them (a
    // separate copy of the path, so the common one keeps its registers)
    uint32_t k0, kend;
    group_slots(a, 2u, k0, kend);
    if (mpc > DENSE_CELL)
        direct_slot_pair_dense<Acc, KERNEL, COUNT>(a, win, threadIdx.x, k0, kend);
    else
        direct_slot_pair<DIRECT_THREADS, false, Acc, KERNEL, COUNT>(a, win, threadIdx.x, k0, kend);
}

// Resident CTAs per SM the four-target direct kernel's registers are capped
// for (the plain kernels: 5, about 100 registers; the others uncapped).
template <class Acc, int KERNEL>
__host__ __device__ constexpr int direct4_min_blocks()
{
    return (std::is_same<Acc, PlainAcc>::value && (KERNEL == KERNEL_GAUSSIAN || KERNEL == KERNEL_LOWFLOP)) ? 5 : 1;
}

// Four targets per thread: P slots 4p .. 4p + 3.  Each source read feeds
// four targets (two packed pairs), so the L1 reads per evaluation halve
// while the union of four windows adds evaluations -- the better trade at
// high occupancy (32 per cell), the worse at low.  Four slots lie in one
// X-row of one system unless some are sentinels (every row ends in
// ROW_PADS of them), which repeat a real target and store nothing.  Grids
// with dense cells take the slot pairs' dense path.
template <class Acc, int KERNEL, bool COUNT = false>
__global__ void __launch_bounds__(DIRECT_THREADS, (direct4_min_blocks<Acc, KERNEL>()))
    k_interact_direct4(InteractArgs a)
{
    __shared__ uint32_t win[20][DIRECT_THREADS];  // 9 windows (lo, hi) + one spare read after the last
    pdl_trigger();
    pdl_wait();  // the binning (or the previous interaction) has completed
    // keep the work counters of the tiled launches in step (see k_interact_tiled)
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctrl->work[(a.seq + 1u) & 1u] = 0u;
    // both control words in flight together, per thread (a per-CTA read
    // and barrier, cta_ctrl_words, measured 1 % slower here: the
    // evaluation hides these reads)
    const uint32_t err = load_error(a.ctrl);
    const uint32_t mpc = *((volatile const uint32_t*)&a.ctrl->max_per_cell);
    if (err) return;
    uint32_t k0, kend;
    group_slots(a, 4u, k0, kend);
    if (k0 >= kend) return;
    if (mpc > DENSE_CELL) {
        direct_slot_pair_dense<Acc, KERNEL, COUNT>(a, win, threadIdx.x, k0, kend);
        direct_slot_pair_dense<Acc, KERNEL, COUNT>(a, win, threadIdx.x, k0 + 2u, kend);
        return;
    }
    constexpr uint32_t NONE = 0xffffffffu;
    float4 t[4];
    bool v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        t[k] = k0 + k < kend ? __ldg(a.P + k0 + k) : make_float4(0.f, 0.f, 0.f, __uint_as_float(NONE));
        v[k] = __float_as_uint(t[k].w) != NONE;
    }
    if (!(v[0] || v[1] || v[2] || v[3])) return;
    const float4 tf = v[0] ? t[0] : (v[1] ? t[1] : (v[2] ? t[2] : t[3]));
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (!v[k]) t[k] = tf;
    // the system of the targets: from a stable slot (= sorted index)
    const int sid = a.sy.S == 1 ? 0 : find_system(a.sy.pbase, a.sy.S, __float_as_uint(tf.w));
    const SysDesc& d = a.sy.sys[sid];
    const Grid& g = d.g;
    int cx[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) cx[k] = axis_cell(t[k].x, g.lo[0], g.inv_w[0], g.n[0]);
    const int cy = axis_cell(tf.y, g.lo[1], g.inv_w[1], g.n[1]);
    const int cz = axis_cell(tf.z, g.lo[2], g.inv_w[2], g.n[2]);
    const KParams kp = kparams(a, sid);
    Sums<Acc, KERNEL> r[4];
    const uint32_t slots =
        direct_group<DIRECT_THREADS, 4, false, Acc, KERNEL, COUNT>(a, d, win, threadIdx.x, t, cx, cy, cz, kp, r);
    add_evals<COUNT>(a, (unsigned long long)slots * ((v[0] ? 1u : 0u) + (v[1] ? 1u : 0u) + (v[2] ? 1u : 0u) +
                                              (v[3] ? 1u : 0u)));
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (v[k]) store_out(a, __float_as_uint(t[k].w), r[k]);
}

// The forms with a counting copy of the direct kernels (PI_OPT_COUNT_EVALS).
template <class Acc, int KERNEL>
constexpr bool counted_form()
{
    return std::is_same<Acc, PlainAcc>::value && (KERNEL == KERNEL_GAUSSIAN || KERNEL == KERNEL_GAUSSIAN_FINE);
}

// Blocks of a direct launch: over all of P, or a.range_blocks for a launch
// over a list of ranges (the host deals the blocks out range by range).
inline unsigned direct_grid(const InteractArgs& a, uint64_t per)
{
    if (a.ranges) return a.range_blocks;
    const uint64_t groups = ((uint64_t)a.np + per - 1) / per;
    return (unsigned)((groups + DIRECT_THREADS - 1) / DIRECT_THREADS);
}

template <class Acc, int KERNEL>
void launch_direct4_one(const InteractArgs& a, cudaStream_t s)
{
    // an error is left for cudaGetLastError
    // the counting copy exists for the plain Gaussian sums (the windows, and
    // so the count, do not depend on the kernel K or the precision)
    if constexpr (counted_form<Acc, KERNEL>()) {
        if (a.count_evals) {
            (void)launch_dependent(k_interact_direct4<Acc, KERNEL, true>, dim3(direct_grid(a, 4)),
                                   dim3(DIRECT_THREADS), 0, s, a);
            return;
        }
    }
    (void)launch_dependent(k_interact_direct4<Acc, KERNEL>, dim3(direct_grid(a, 4)), dim3(DIRECT_THREADS), 0, s, a);
}

template <class Acc, int KERNEL>
void launch_direct_one(const InteractArgs& a, cudaStream_t s)
{
    // an error is left for cudaGetLastError
    if constexpr (counted_form<Acc, KERNEL>()) {
        if (a.count_evals) {
            (void)launch_dependent(k_interact_direct<Acc, KERNEL, true>, dim3(direct_grid(a, 2)),
                                   dim3(DIRECT_THREADS), 0, s, a);
            return;
        }
    }
    (void)launch_dependent(k_interact_direct<Acc, KERNEL>, dim3(direct_grid(a, 2)), dim3(DIRECT_THREADS), 0, s, a);
}

template <class Acc>
cudaError_t launch_ppnl_acc(const InteractArgs& a, cudaStream_t s)
{
    const dim3 blocks((unsigned)((a.n + 127) / 128)), threads(128);
    switch (a.kernel) {
        case KERNEL_LJ: return launch_dependent(k_interact_ppnl<Acc, KERNEL_LJ>, blocks, threads, 0, s, a);
        case KERNEL_LOWFLOP: return launch_dependent(k_interact_ppnl<Acc, KERNEL_LOWFLOP>, blocks, threads, 0, s, a);
        case KERNEL_HIGHFLOP: return launch_dependent(k_interact_ppnl<Acc, KERNEL_HIGHFLOP>, blocks, threads, 0, s, a);
        case KERNEL_GAUSSIAN_FINE:
            return launch_dependent(k_interact_ppnl<Acc, KERNEL_GAUSSIAN_FINE>, blocks, threads, 0, s, a);
        default: return launch_dependent(k_interact_ppnl<Acc, KERNEL_GAUSSIAN>, blocks, threads, 0, s, a);
    }
}

template <class T, class Acc, int KERNEL>
void launch_tiled_one(const InteractArgs& a, unsigned grid, cudaStream_t s)
{
    // an error is left for cudaGetLastError
    (void)launch_dependent(k_interact_tiled<T, Acc, KERNEL>, dim3(grid), dim3(T::NT), sizeof(Smem<T>), s, a);
}

template <class T, class Acc, int KERNEL>
void launch_ws_one(const InteractArgs& a, unsigned grid, cudaStream_t s)
{
    // an error is left for cudaGetLastError
    (void)launch_dependent(k_interact_ws<T, Acc, KERNEL>, dim3(grid), dim3(T::THREADS), sizeof(WsSmem<T>), s, a);
}

template <class Acc>
cudaError_t launch_tiled_acc(const InteractArgs& a, int tile, const int* per_sm, int num_sms,
                             cudaStream_t s)
{
    // the comparator kernels and the fine Gaussian run on the direct kernels
    // or the 128-thread shape
    if (a.kernel != KERNEL_GAUSSIAN && tile != 5 && tile != 6) tile = 2;
    uint64_t grid = (uint64_t)num_sms * (uint64_t)(per_sm[tile] < 1 ? 1 : per_sm[tile]);
    if (grid > a.work) grid = a.work;
    if (grid < 1) grid = 1;
    const unsigned g = (unsigned)grid;
    switch (a.kernel) {
        case KERNEL_LJ:
            tile == 5   ? launch_direct_one<Acc, KERNEL_LJ>(a, s)
            : tile == 6 ? launch_direct4_one<Acc, KERNEL_LJ>(a, s)
                        : launch_tiled_one<TileL, Acc, KERNEL_LJ>(a, g, s);
            break;
        case KERNEL_LOWFLOP:
            tile == 5   ? launch_direct_one<Acc, KERNEL_LOWFLOP>(a, s)
            : tile == 6 ? launch_direct4_one<Acc, KERNEL_LOWFLOP>(a, s)
                        : launch_tiled_one<TileL, Acc, KERNEL_LOWFLOP>(a, g, s);
            break;
        case KERNEL_HIGHFLOP:
            tile == 5   ? launch_direct_one<Acc, KERNEL_HIGHFLOP>(a, s)
            : tile == 6 ? launch_direct4_one<Acc, KERNEL_HIGHFLOP>(a, s)
                        : launch_tiled_one<TileL, Acc, KERNEL_HIGHFLOP>(a, g, s);
            break;
        case KERNEL_GAUSSIAN_FINE:
            tile == 5   ? launch_direct_one<Acc, KERNEL_GAUSSIAN_FINE>(a, s)
            : tile == 6 ? launch_direct4_one<Acc, KERNEL_GAUSSIAN_FINE>(a, s)
                        : launch_tiled_one<TileL, Acc, KERNEL_GAUSSIAN_FINE>(a, g, s);
            break;
        default:
            switch (tile) {
                case 0: launch_tiled_one<TileS, Acc, KERNEL_GAUSSIAN>(a, g, s); break;
                case 1: launch_tiled_one<TileM, Acc, KERNEL_GAUSSIAN>(a, g, s); break;
                case 2: launch_tiled_one<TileL, Acc, KERNEL_GAUSSIAN>(a, g, s); break;
                case 4: launch_ws_one<Ws8, Acc, KERNEL_GAUSSIAN>(a, g, s); break;
                case 5: launch_direct_one<Acc, KERNEL_GAUSSIAN>(a, s); break;
                case 6: launch_direct4_one<Acc, KERNEL_GAUSSIAN>(a, s); break;
                default: launch_ws_one<Ws4, Acc, KERNEL_GAUSSIAN>(a, g, s); break;
            }
            break;
    }
    return cudaGetLastError();
}

// Allows the shape's dynamic shared memory (above the 48 KB default for the
// largest shape) and returns its resident CTAs per SM.
template <class T, class Acc>
cudaError_t ws_occupancy_of(int* per_sm)
{
    auto fn = k_interact_ws<T, Acc, KERNEL_GAUSSIAN>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(WsSmem<T>));
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, T::THREADS, sizeof(WsSmem<T>));
}

template <class T, class Acc>
cudaError_t occupancy_of(int* per_sm)
{
    auto fn = k_interact_tiled<T, Acc, KERNEL_GAUSSIAN>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem<T>));
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, T::NT, sizeof(Smem<T>));
}

}  // namespace

cudaError_t launch_interact_ppnl(const InteractArgs& a, bool kahan, int num_sms, cudaStream_t s,
                                 int* launches)
{
    (void)num_sms;
    *launches += 1;
    return kahan ? launch_ppnl_acc<KahanAcc>(a, s) : launch_ppnl_acc<PlainAcc>(a, s);
}

template <class Acc>
cudaError_t tiled_occupancy_acc(int* per_sm)
{
    cudaError_t e;
    if ((e = occupancy_of<TileS, Acc>(&per_sm[0])) != cudaSuccess) return e;
    if ((e = occupancy_of<TileM, Acc>(&per_sm[1])) != cudaSuccess) return e;
    if ((e = occupancy_of<TileL, Acc>(&per_sm[2])) != cudaSuccess) return e;
    if ((e = ws_occupancy_of<Ws4, Acc>(&per_sm[3])) != cudaSuccess) return e;
    if ((e = ws_occupancy_of<Ws8, Acc>(&per_sm[4])) != cudaSuccess) return e;
    per_sm[5] = 1;  // the direct kernels launch one thread per two or four targets
    per_sm[6] = 1;
    // the comparator kernels run with the 128-thread shape: allow its shared memory
    constexpr int bytes = (int)sizeof(Smem<TileL>);
    if ((e = cudaFuncSetAttribute(k_interact_tiled<TileL, Acc, KERNEL_LJ>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_interact_tiled<TileL, Acc, KERNEL_LOWFLOP>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_interact_tiled<TileL, Acc, KERNEL_GAUSSIAN_FINE>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(k_interact_tiled<TileL, Acc, KERNEL_HIGHFLOP>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t tiled_occupancy(bool kahan, int* per_sm)
{
    static_assert(NUM_TILES == 7, "one occupancy entry per tile shape");
    return kahan ? tiled_occupancy_acc<KahanAcc>(per_sm) : tiled_occupancy_acc<PlainAcc>(per_sm);
}

cudaError_t launch_interact_tiled(const InteractArgs& a, bool kahan, int num_sms, const int* per_sm,
                                  int tile, cudaStream_t s, int* launches)
{
    *launches += 1;
    return kahan ? launch_tiled_acc<KahanAcc>(a, tile, per_sm, num_sms, s)
                 : launch_tiled_acc<PlainAcc>(a, tile, per_sm, num_sms, s);
}

}  // namespace pi
