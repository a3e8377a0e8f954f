// pi_bin.cu -- binning kernels (arXiv 2406.16091, Sec. 2 and Fig. 1).
//
//   k_zero       clears the control block and the per-cell counts
//   k_hist       a1 + a2: cell index of each particle (float4 SoA loads) and an
//                atomic histogram, one atomicAdd per particle; the value it
//                returns is kept as a provisional slot inside the cell
//   k_scan       a3: single-pass exclusive scan over the C+1 counts with
//                decoupled lookback (dynamic tile ticket, bounded waits), and
//                M_C, the largest count (Sec. 5.1 keeps it during the scan)
//   k_scatter    a4, first half: each particle (and its position) to its
//                provisional slot (the paper's atomic scatter, whose order
//                inside a cell is arbitrary)
//   k_stabilise  a4, second half: rank each particle among its cell's members
//                by input index, which makes the order stable; write the
//                sorted positions, the row-padded x-ordered copy P that the
//                interaction reads, and each cell's x-sub-bin starts
//
// All kernels are HBM- or L2-bound integer work; none uses tensor cores.
#include <algorithm>
#include <mutex>

#include "pi_internal.cuh"

namespace pi {

namespace {

constexpr unsigned FULL = 0xffffffffu;

template <int NB>
__global__ void k_zero(ZeroArgs<NB> z)
{
    pdl_trigger();
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    uint4* p4 = reinterpret_cast<uint4*>(z.p);
    size_t n4 = z.n_words / 4;
    for (size_t k = i; k < n4; k += stride) p4[k] = make_uint4(0, 0, 0, 0);
    for (size_t k = n4 * 4 + i; k < z.n_words; k += stride) z.p[k] = 0;
    for (size_t k = i; k < (size_t)z.nb; k += stride) z.pbase[k] = z.vals[k];
}

// Particles per lane of k_hist (a multiple of 4: float4 loads and stores).
constexpr int HIST_PER_LANE = 4;

// a1 + a2.  Each lane owns a group of HIST_PER_LANE consecutive particles,
// loaded as float4s per component when the arrays are 16-byte aligned, so
// that all of its atomics are in flight together.  The system of each
// particle comes from the particle bases; its cell is offset by the system's
// first cell.
__global__ void __launch_bounds__(256) k_hist(const float* __restrict__ x,
                                              const float* __restrict__ y,
                                              const float* __restrict__ z, uint32_t n, Systems sy,
                                              uint32_t* __restrict__ counts,
                                              uint32_t* __restrict__ cell_out,
                                              uint32_t* __restrict__ rank_out,
                                              Ctrl* __restrict__ ctrl, int vec)
{
    constexpr int HP = HIST_PER_LANE, HV = HP / 4;
    pdl_trigger();
    const unsigned lane = threadIdx.x & 31u;
    const uint32_t groups = (n + HP - 1u) / HP;
    const uint32_t stride = gridDim.x * blockDim.x;
    bool all_ok = true;
    for (uint32_t g0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); g0 < groups; g0 += stride) {
        const uint32_t grp = g0 + lane;
        const uint32_t i0 = grp * HP;
        float px[HP], py[HP], pz[HP];
        bool valid[HP];
        const bool full = (grp < groups) && (i0 + HP <= n);
        if (full && vec) {
#pragma unroll
            for (int v = 0; v < HV; ++v) {
                const float4 a = __ldcs(reinterpret_cast<const float4*>(x) + grp * HV + v);
                const float4 b = __ldcs(reinterpret_cast<const float4*>(y) + grp * HV + v);
                const float4 c = __ldcs(reinterpret_cast<const float4*>(z) + grp * HV + v);
                px[4 * v] = a.x; px[4 * v + 1] = a.y; px[4 * v + 2] = a.z; px[4 * v + 3] = a.w;
                py[4 * v] = b.x; py[4 * v + 1] = b.y; py[4 * v + 2] = b.z; py[4 * v + 3] = b.w;
                pz[4 * v] = c.x; pz[4 * v + 1] = c.y; pz[4 * v + 2] = c.z; pz[4 * v + 3] = c.w;
            }
#pragma unroll
            for (int j = 0; j < HP; ++j) valid[j] = true;
        } else {
#pragma unroll
            for (int j = 0; j < HP; ++j) {
                const uint32_t i = i0 + j;
                valid[j] = (grp < groups) && (i < n);
                px[j] = valid[j] ? x[i] : 0.f;
                py[j] = valid[j] ? y[i] : 0.f;
                pz[j] = valid[j] ? z[i] : 0.f;
            }
        }
        // the positions are the caller's input, written before k_zero started;
        // the particle bases and the counts are k_zero's
        pdl_wait();
        int s = (sy.S == 1 || grp >= groups) ? 0 : find_system(sy.pbase, sy.S, i0);
        // all cells, then all atomics: the atomics of one lane are in flight
        // together.  Particles come in no spatial order, so a warp almost
        // never holds two of one cell: no warp aggregation.
        uint32_t cell[HP], rank[HP];
#pragma unroll
        for (int j = 0; j < HP; ++j) {
            if (sy.S > 1 && valid[j])
                while (s + 1 < sy.S && i0 + j >= __ldg(sy.pbase + s + 1)) ++s;
            const SysDesc& d = sy.sys[s];
            bool ok = true;
            cell[j] = cell_of(px[j], py[j], pz[j], d.g, ok) + d.cell_base;
            all_ok &= ok | !valid[j];
        }
#ifdef PI_CHECK
        const uint32_t c_all = __ldg(sy.cbase + sy.S);
#pragma unroll
        for (int j = 0; j < HP; ++j) valid[j] = valid[j] && PI_BOUNDS(ctrl, cell[j], c_all, CS_HIST_COUNTS);
#endif
#pragma unroll
        for (int j = 0; j < HP; ++j) rank[j] = valid[j] ? atomicAdd(&counts[cell[j]], 1u) : 0u;
        if (full) {
#pragma unroll
            for (int v = 0; v < HV; ++v) {
                reinterpret_cast<uint4*>(cell_out)[grp * HV + v] =
                    make_uint4(cell[4 * v], cell[4 * v + 1], cell[4 * v + 2], cell[4 * v + 3]);
                reinterpret_cast<uint4*>(rank_out)[grp * HV + v] =
                    make_uint4(rank[4 * v], rank[4 * v + 1], rank[4 * v + 2], rank[4 * v + 3]);
            }
        } else {
#pragma unroll
            for (int j = 0; j < HP; ++j)
                if (valid[j]) {
                    cell_out[i0 + j] = cell[j];
                    rank_out[i0 + j] = rank[j];
                }
        }
    }
    if (!all_ok) atomicOr(&ctrl->error, ERR_OUT_OF_BOX);
}

// ---- a3: decoupled-lookback exclusive scan --------------------------------
//
// Tile descriptor (64 bits): value in bits 0..31, flag in bits 32..33
// (1 = tile aggregate, 2 = inclusive prefix), launch epoch in bits 34..63.
// A descriptor from another launch has another epoch and reads as "not
// ready", so the array never needs clearing between launches.

constexpr uint32_t FLAG_AGG = 1u, FLAG_INCL = 2u;

__device__ __forceinline__ unsigned long long pack_status(uint32_t epoch, uint32_t flag, uint32_t v)
{
    return ((unsigned long long)epoch << 34) | ((unsigned long long)flag << 32) | v;
}

__device__ __forceinline__ void publish(unsigned long long* p, unsigned long long w)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}

__device__ __forceinline__ unsigned long long peek(const unsigned long long* p)
{
    unsigned long long w;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
    return w;
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan(const uint32_t* __restrict__ counts, uint32_t C,
                                                       uint32_t* __restrict__ offsets,
                                                       unsigned long long* __restrict__ status,
                                                       Ctrl* __restrict__ ctrl, uint32_t epoch,
                                                       uint64_t wait_limit_ns, int withhold_first, int track_max,
                                                       int ticket_slot)
{
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_warp_sum[SCAN_THREADS / 32];
    __shared__ uint32_t s_warp_max[SCAN_THREADS / 32];
    __shared__ uint32_t s_prefix;

    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    pdl_trigger();
    pdl_wait();
    if (threadIdx.x == 0) s_tile = atomicAdd(ticket_slot ? &ctrl->tickets[ticket_slot - 1] : &ctrl->ticket, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint64_t items = (uint64_t)C + 1;  // item C is a zero count -> offsets[C] = total
    if (!PI_BOUNDS(ctrl, tile, (items + SCAN_TILE - 1) / SCAN_TILE, CS_SCAN_TILE)) return;
    const uint64_t my0 = (uint64_t)tile * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_ITEMS;

    uint32_t v[SCAN_ITEMS];
    if (my0 + SCAN_ITEMS <= C) {
        const uint4* src = reinterpret_cast<const uint4*>(counts + my0);
#pragma unroll
        for (int q = 0; q < SCAN_ITEMS / 4; ++q) {
            uint4 u = src[q];
            v[4 * q] = u.x; v[4 * q + 1] = u.y; v[4 * q + 2] = u.z; v[4 * q + 3] = u.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) v[k] = (my0 + k < C) ? counts[my0 + k] : 0u;
    }
    uint32_t run = 0, mx = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        uint32_t t = v[k];
        mx = max(mx, t);
        v[k] = run;  // exclusive inside the thread
        run += t;
    }
    // block-wide exclusive scan of the per-thread totals
    uint32_t incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(FULL, incl, o);
        if (lane >= (unsigned)o) incl += t;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(FULL, mx, o));
    if (lane == 31) s_warp_sum[warp] = incl;
    if (lane == 0) s_warp_max[warp] = mx;
    __syncthreads();
    uint32_t warp_excl = 0, tile_sum = 0, tile_max = 0;
#pragma unroll
    for (int w = 0; w < SCAN_THREADS / 32; ++w) {
        uint32_t t = s_warp_sum[w];
        if (w < (int)warp) warp_excl += t;
        tile_sum += t;
        tile_max = max(tile_max, s_warp_max[w]);
    }
    const uint32_t thread_excl = warp_excl + incl - run;

    if (warp == 0) {
        uint32_t prefix = 0;
        if (tile == 0) {
            if (lane == 0 && !withhold_first) publish(&status[0], pack_status(epoch, FLAG_INCL, tile_sum));
        } else {
            if (lane == 0) publish(&status[tile], pack_status(epoch, FLAG_AGG, tile_sum));
            const uint64_t t0 = global_ns();
            int64_t p = (int64_t)tile - 1;
            bool timed_out = false;
            for (;;) {
                const int64_t q = p - (int64_t)lane;
                uint32_t flag = FLAG_INCL, val = 0;
                for (;;) {
                    if (q >= 0) {
                        unsigned long long w = peek(&status[q]);
                        flag = ((uint32_t)(w >> 34) == epoch) ? (uint32_t)(w >> 32) & 3u : 0u;
                        val = (uint32_t)w;
                    }
                    if (__ballot_sync(FULL, flag == 0u) == 0u) break;
                    const bool late = __shfl_sync(FULL, (global_ns() - t0) > wait_limit_ns, 0);
                    if (late) { timed_out = true; break; }
                    __nanosleep(64);
                }
                if (timed_out) break;
                const unsigned incl_mask = __ballot_sync(FULL, flag == FLAG_INCL);
                const int stop = incl_mask ? __ffs(incl_mask) - 1 : 31;
                prefix += warp_sum((int)lane <= stop ? val : 0u);
                if (incl_mask) break;
                p -= 32;
            }
            if (lane == 0) {
                if (timed_out) atomicOr(&ctrl->error, ERR_TIMEOUT);
                // publish even after a timeout so that later tiles finish quickly
                publish(&status[tile], pack_status(epoch, FLAG_INCL, prefix + tile_sum));
            }
        }
        if (lane == 0) {
            s_prefix = prefix;
            if (tile_max && track_max) atomicMax(&ctrl->max_per_cell, tile_max);
        }
    }
    __syncthreads();
    const uint32_t base = s_prefix + thread_excl;
    if (my0 + SCAN_ITEMS <= items) {
        uint4* dst = reinterpret_cast<uint4*>(offsets + my0);
#pragma unroll
        for (int q = 0; q < SCAN_ITEMS / 4; ++q)
            dst[q] = make_uint4(base + v[4 * q], base + v[4 * q + 1], base + v[4 * q + 2],
                                base + v[4 * q + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k)
            if (my0 + k < items) offsets[my0 + k] = base + v[k];
    }
}

// ---- a4 ---------------------------------------------------------------------

// One record as a single 256-bit store: a whole 32-byte DRAM sector, so the
// random write needs no read of the rest of the sector.
__device__ __forceinline__ void store_rec(Rec* dst, float x, uint32_t i, uint32_t t_lo, uint32_t t_hi, float y,
                                          float z, uint32_t c)
{
    asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(dst),
                 "r"(__float_as_uint(x)), "r"(i), "r"(t_lo), "r"(t_hi), "r"(__float_as_uint(y)),
                 "r"(__float_as_uint(z)), "r"(c), "r"(0u)
                 : "memory");
}

__device__ __forceinline__ Rec load_rec(const Rec* src)
{
    Rec r;
    uint32_t x, y, z;
    asm volatile("ld.global.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(x), "=r"(r.i), "=r"(r.t_lo), "=r"(r.t_hi), "=r"(y), "=r"(z), "=r"(r.c), "=r"(r.pad)
                 : "l"(src));
    r.x = __uint_as_float(x);
    r.y = __uint_as_float(y);
    r.z = __uint_as_float(z);
    return r;
}

// The x-sub-bin thermometer of a particle at x in cell c_local of grid g
// (see Rec and x_sub_bin).
__device__ __forceinline__ uint2 sub_bin_thermometer(float x, uint32_t c_local, const Grid& g)
{
    return thermometer(x_sub_bin(x, c_local, g));
}

// a4, first half: each particle to its provisional slot offsets[cell] +
// rank.  Each lane owns a group of 4 consecutive particles (vector loads when
// the inputs are 16-byte aligned), so four records are in flight at once.
__global__ void __launch_bounds__(256) k_scatter(const uint32_t* __restrict__ cell,
                                                 const uint32_t* __restrict__ rank,
                                                 const float* __restrict__ x,
                                                 const float* __restrict__ y,
                                                 const float* __restrict__ z, uint32_t n, Systems sy,
                                                 const uint32_t* __restrict__ offsets,
                                                 Rec* __restrict__ rec, Ctrl* __restrict__ ctrl,
                                                 int vec)
{
    pdl_trigger();
    pdl_wait();
    if (cta_error(ctrl)) return;
    bool bad = false;
    const uint32_t groups = (n + 3u) / 4u;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < groups; g += gridDim.x * blockDim.x) {
        const uint32_t i0 = 4u * g;
        uint32_t c[4], r[4];
        float px[4], py[4], pz[4];
        bool valid[4];
        if (i0 + 4u <= n) {
            const uint4 cc = reinterpret_cast<const uint4*>(cell)[g];
            const uint4 rr = reinterpret_cast<const uint4*>(rank)[g];
            c[0] = cc.x; c[1] = cc.y; c[2] = cc.z; c[3] = cc.w;
            r[0] = rr.x; r[1] = rr.y; r[2] = rr.z; r[3] = rr.w;
            if (vec) {
                const float4 a = __ldcs(reinterpret_cast<const float4*>(x) + g);
                const float4 b = __ldcs(reinterpret_cast<const float4*>(y) + g);
                const float4 d = __ldcs(reinterpret_cast<const float4*>(z) + g);
                px[0] = a.x; px[1] = a.y; px[2] = a.z; px[3] = a.w;
                py[0] = b.x; py[1] = b.y; py[2] = b.z; py[3] = b.w;
                pz[0] = d.x; pz[1] = d.y; pz[2] = d.z; pz[3] = d.w;
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    px[j] = x[i0 + j];
                    py[j] = y[i0 + j];
                    pz[j] = z[i0 + j];
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) valid[j] = true;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t i = i0 + j;
                valid[j] = i < n;
                c[j] = valid[j] ? cell[i] : 0u;
                r[j] = valid[j] ? rank[i] : 0u;
                px[j] = valid[j] ? x[i] : 0.f;
                py[j] = valid[j] ? y[i] : 0.f;
                pz[j] = valid[j] ? z[i] : 0.f;
            }
        }
        // rank < count holds by the atomic's semantics, so the slot lies in
        // the cell's range; the test against n only keeps a corrupted rank
        // from writing outside the records
        uint32_t lo[4];
#ifdef PI_CHECK
        const uint32_t c_all = __ldg(sy.cbase + sy.S);
#pragma unroll
        for (int j = 0; j < 4; ++j) valid[j] = valid[j] && PI_BOUNDS(ctrl, c[j], c_all, CS_SCATTER_REC);
#endif
#pragma unroll
        for (int j = 0; j < 4; ++j) lo[j] = valid[j] ? offsets[c[j]] : 0u;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!valid[j]) continue;
            const int sid = sy.S == 1 ? 0 : find_system(sy.cbase, sy.S, c[j]);
            const SysDesc& d = sy.sys[sid];
            const uint2 t = sub_bin_thermometer(px[j], c[j] - d.cell_base, d.g);
            const uint32_t slot = lo[j] + r[j];
            if (slot < n) store_rec(rec + slot, px[j], i0 + j, t.x, t.y, py[j], pz[j], c[j]);
            else bad = true;
        }
    }
    if (bad) atomicOr(&ctrl->error, ERR_CAPACITY);
}

// a4, second half, one thread per provisional slot k.  The members of k's
// cell sit contiguously in rec, so every member read is coalesced across the
// warp.  From them the thread computes
//   - the stable rank: members with a smaller input index (input order
//     inside the cell), and writes perm, sx, sy, sz at that slot;
//   - the x-rank: members with smaller x (ties by input index), and writes
//     P[s0 + x-rank + ROW_PADS * row] = (x, y, z, stable slot).  The cells
//     of an X-row are contiguous and monotone in x, so every X-row of P is
//     sorted by x as a whole -- the tiled interaction stages such rows --
//     and followed by ROW_PADS sentinel slots (written here too);
//   - (the member of x-rank 0 only) xbins[c]: byte b - 1 (b = 1 .. XSUB - 1)
//     = members whose x-sub-bin is < b, the sum of the members' thermometers
//     (see Rec); byte 7 holds flags: XBIN_COARSE when the cell has more
//     than 255 members (bytes 0..6 then 0: every sub-bin starts at the
//     cell), XBIN_DENSE when it has more than DENSE_CELL.
__global__ void __launch_bounds__(256) k_stabilise(const Rec* __restrict__ rec, uint32_t n,
                                                   Systems sy, const uint32_t* __restrict__ offsets,
                                                   uint32_t* __restrict__ perm,
                                                   float* __restrict__ sx, float* __restrict__ sy_out,
                                                   float* __restrict__ sz, float4* __restrict__ P,
                                                   uint2* __restrict__ xbins,
                                                   Ctrl* __restrict__ ctrl)
{
    pdl_trigger();
    pdl_wait();
    if (cta_error(ctrl)) return;
    bool bad = false;
    const uint32_t C = __ldg(sy.cbase + sy.S);
    // the sentinel slots after every X-row of P: a particle far from every
    // other one (finite coordinates, so its pair terms are exact zeros)
    const uint32_t rows = __ldg(sy.rbase + sy.S);
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
        const int sid = sy.S == 1 ? 0 : find_system(sy.rbase, sy.S, r);
        const SysDesc& d = sy.sys[sid];
        const uint32_t end_cell = d.cell_base + (r - d.row_base + 1u) * (uint32_t)d.g.n[0];
        const uint32_t pos = offsets[end_cell] + ROW_PADS * r;
        if (!PI_BOUNDS(ctrl, pos + ROW_PADS - 1u, (uint64_t)n + ROW_PADS * (uint64_t)rows, CS_STAB_OUT)) continue;
#pragma unroll
        for (int k = 0; k < ROW_PADS; ++k)
            P[pos + k] = make_float4(1e18f, 1e18f, 1e18f, __uint_as_float(0xffffffffu));
    }
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const Rec me = load_rec(rec + k);
        const uint32_t i = me.i, c = me.c;
        if (i >= n || c >= C) { bad = true; continue; }
        const uint32_t s0 = offsets[c], s1 = offsets[c + 1];
        if (k < s0 || k >= s1) { bad = true; continue; }
        if (!PI_BOUNDS(ctrl, s1 - 1u, n, CS_STAB_MEMBER)) continue;
        // stable rank, x-rank and the sum of the members' sub-bin
        // thermometers (byte b - 1 = members whose sub-bin is < b)
        uint32_t r = 0, xr = 0, lt_lo = 0, lt_hi = 0;
        for (uint32_t q = s0; q < s1; ++q) {
            const uint4 m = *reinterpret_cast<const uint4*>(rec + q);  // (x, input index, thermometer)
            const float xq = __uint_as_float(m.x);
            const uint32_t j = m.y;
            r += (j < i) ? 1u : 0u;
            xr += (xq < me.x || (xq == me.x && j < i)) ? 1u : 0u;
            lt_lo += m.z;
            lt_hi += m.w;
        }
        const uint32_t dst = s0 + r;
        if (!PI_BOUNDS(ctrl, dst, n, CS_STAB_OUT)) continue;
        perm[dst] = i;
        sx[dst] = me.x;
        sy_out[dst] = me.y;
        sz[dst] = me.z;
        const int sid = sy.S == 1 ? 0 : find_system(sy.cbase, sy.S, c);
        const SysDesc& d = sy.sys[sid];
        const uint32_t row = d.row_base + (c - d.cell_base) / (uint32_t)d.g.n[0];
        if (!PI_BOUNDS(ctrl, s0 + xr + ROW_PADS * row, (uint64_t)n + ROW_PADS * (uint64_t)rows, CS_STAB_OUT)) continue;
        P[s0 + xr + ROW_PADS * row] = make_float4(me.x, me.y, me.z, __uint_as_float(dst));
        // the first member in x order writes the cell's sub-bin starts; the
        // byte sums are exact up to 255 members, larger cells are flagged
        static_assert(XSUB == 8, "xbins packs 7 sub-bin starts and a flag into 8 bytes");
        if (xr == 0) {
            const uint32_t m = s1 - s0;
            xbins[c] = m > 255u ? make_uint2(0u, XBIN_COARSE << 24)
                                : make_uint2(lt_lo, lt_hi | (m > DENSE_CELL ? XBIN_DENSE << 24 : 0u));
        }
    }
    if (bad) atomicOr(&ctrl->error, ERR_CAPACITY);
}

// Resident CTAs per SM of a binning kernel (256 threads, no dynamic shared
// memory) on the current device, queried once per device and kernel.
template <class F>
int resident_per_sm(F* fn, int slot)
{
    constexpr int MAXDEV = 64, SLOTS = 4;
    static std::mutex mu;
    static int cache[MAXDEV][SLOTS] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAXDEV) return 4;
    std::lock_guard<std::mutex> lock(mu);
    if (cache[dev][slot] == 0) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, 256, 0) != cudaSuccess || b < 1) b = 4;
        cache[dev][slot] = b;
    }
    return cache[dev][slot];
}

inline int grid_for(uint64_t work, int threads, int num_sms, int per_sm)
{
    uint64_t b = (work + threads - 1) / threads;
    uint64_t cap = (uint64_t)num_sms * per_sm;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

template <int NB>
cudaError_t launch_zero_nb(uint32_t* p, size_t n_words, uint32_t* pbase, const uint32_t* vals, int nb,
                           cudaStream_t s)
{
    ZeroArgs<NB> z;
    z.p = p;
    z.n_words = n_words;
    z.pbase = pbase;
    z.nb = nb;
    for (int k = 0; k < nb; ++k) z.vals[k] = vals[k];
    int blocks = (int)((n_words / 4 + 255) / 256);
    blocks = blocks < 1 ? 1 : (blocks > 1184 ? 1184 : blocks);
    k_zero<NB><<<blocks, 256, 0, s>>>(z);
    return cudaGetLastError();
}

cudaError_t launch_zero(uint32_t* p, size_t n_words, uint32_t* pbase, const uint32_t* vals, int nb,
                        cudaStream_t s)
{
    if (nb <= 8) return launch_zero_nb<8>(p, n_words, pbase, vals, nb, s);
    return launch_zero_nb<MAX_SYSTEMS + 1>(p, n_words, pbase, vals, nb, s);
}

cudaError_t launch_hist(const float* x, const float* y, const float* z, uint32_t n,
                        const Systems& sy, uint32_t* counts, uint32_t* cell, uint32_t* rank,
                        Ctrl* ctrl, int num_sms, cudaStream_t s)
{
    const int vec = ((((uintptr_t)x) | ((uintptr_t)y) | ((uintptr_t)z)) & 15u) == 0;
    const uint64_t groups = ((uint64_t)n + HIST_PER_LANE - 1) / HIST_PER_LANE;
    // exactly the resident CTAs (grid-stride loop): no partial last wave
    return launch_dependent(k_hist, dim3(grid_for(groups, 256, num_sms, resident_per_sm(k_hist, 0))), dim3(256), 0, s,
                            x, y, z, n, sy, counts, cell, rank, ctrl, vec);
}

cudaError_t launch_scan(const uint32_t* counts, uint32_t C, uint32_t* offsets,
                        unsigned long long* status, Ctrl* ctrl, uint32_t epoch,
                        uint64_t wait_limit_ns, int withhold_first, cudaStream_t s, int track_max,
                        int ticket_slot)
{
    if (ticket_slot < 0 || ticket_slot > 3) return cudaErrorInvalidValue;
    const uint64_t tiles = ((uint64_t)C + 1 + SCAN_TILE - 1) / SCAN_TILE;
    return launch_dependent(k_scan, dim3((unsigned)tiles), dim3(SCAN_THREADS), 0, s, counts, C, offsets, status,
                            ctrl, epoch, wait_limit_ns, withhold_first, track_max, ticket_slot);
}

cudaError_t launch_scatter(const uint32_t* cell, const uint32_t* rank, const float* x,
                           const float* y, const float* z, uint32_t n, const Systems& sy,
                           const uint32_t* offsets, Rec* rec, Ctrl* ctrl, int num_sms, cudaStream_t s)
{
    const int vec = ((((uintptr_t)x) | ((uintptr_t)y) | ((uintptr_t)z)) & 15u) == 0;
    const uint64_t groups = ((uint64_t)n + 3) / 4;
    return launch_dependent(k_scatter, dim3(grid_for(groups, 256, num_sms, resident_per_sm(k_scatter, 1))), dim3(256),
                            0, s, cell, rank, x, y, z, n, sy, offsets, rec, ctrl, vec);
}

cudaError_t launch_stabilise(const Rec* rec, uint32_t n, const Systems& sy, const uint32_t* offsets,
                             uint32_t* perm, float* sx, float* sy_out, float* sz, float4* P,
                             uint2* xbins, Ctrl* ctrl, int num_sms, cudaStream_t s)
{
    return launch_dependent(k_stabilise, dim3(grid_for(n, 256, num_sms, resident_per_sm(k_stabilise, 2))), dim3(256),
                            0, s, rec, n, sy, offsets, perm, sx, sy_out, sz, P, xbins, ctrl);
}

namespace {
__global__ void k_set_system(SysDesc* sys, uint32_t* cbase, uint32_t* wbase, uint32_t* rbase, SysDesc d,
                             uint32_t cells, uint32_t work, uint32_t rows)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sys[0] = d;
        cbase[1] = cells;
        wbase[1] = work;
        rbase[1] = rows;
    }
}

struct KscaleArgs {
    float* dst;
    int count;
    float vals[2 * MAX_SYSTEMS];
};

__global__ void k_set_kscale(KscaleArgs k)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k.count; i += gridDim.x * blockDim.x)
        k.dst[i] = k.vals[i];
}
}  // namespace

cudaError_t launch_set_system(SysDesc* sys, uint32_t* cbase, uint32_t* wbase, uint32_t* rbase,
                              const SysDesc& d, uint32_t cells, uint32_t work, uint32_t rows, cudaStream_t s)
{
    k_set_system<<<1, 32, 0, s>>>(sys, cbase, wbase, rbase, d, cells, work, rows);
    return cudaGetLastError();
}

namespace {
constexpr int WORDS_PER_LAUNCH = 4096;
struct WordsArgs {
    uint32_t* dst;
    int count;
    uint32_t vals[WORDS_PER_LAUNCH];
};

__global__ void k_write_words(WordsArgs k)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k.count; i += gridDim.x * blockDim.x)
        k.dst[i] = k.vals[i];
}
}  // namespace

cudaError_t launch_write_words(uint32_t* dst, const uint32_t* vals, size_t count, cudaStream_t s)
{
    for (size_t off = 0; off < count; off += WORDS_PER_LAUNCH) {
        WordsArgs k;
        k.dst = dst + off;
        k.count = (int)std::min<size_t>(WORDS_PER_LAUNCH, count - off);
        for (int i = 0; i < k.count; ++i) k.vals[i] = vals[off + i];
        k_write_words<<<(k.count + 255) / 256, 256, 0, s>>>(k);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_set_kscale(float* kscale, const float* vals, int count, cudaStream_t s)
{
    if (count < 0 || count > 2 * MAX_SYSTEMS) return cudaErrorInvalidValue;
    KscaleArgs k;
    k.dst = kscale;
    k.count = count;
    for (int i = 0; i < count; ++i) k.vals[i] = vals[i];
    k_set_kscale<<<(count + 255) / 256, 256, 0, s>>>(k);
    return cudaGetLastError();
}

}  // namespace pi
