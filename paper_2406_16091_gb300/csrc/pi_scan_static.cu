// pi_scan_static.cu -- the exclusive scan of per-cell counts (the a3 kernel,
// k_scan) for callers that cannot allocate device memory.
//
// The scan needs scratch: a control block (tile ticket, error bits, M_C) and
// one lookback descriptor per 4096-count tile.  pi_bin keeps that scratch in
// the arena pi_create allocates.  This entry point keeps it instead in one
// file-scope __device__ array of fixed size, so it calls no cudaMalloc, no
// cudaFree and no allocating library routine; the caller passes the counts
// and the output offsets.
//
// The array lives in every GPU that loads the library until the process
// exits.  Host code cannot use the array's name as a device address (it
// names a host-side stand-in), so the first call on each device looks the
// address up with cudaGetSymbolAddress, with that device current, and caches
// it; later calls on that device reuse the cached address.
#include <cstdio>
#include <mutex>

#include "pi.h"
#include "pi_internal.cuh"

namespace {

constexpr int64_t NOALLOC_MAX_CELLS = (int64_t)1 << 24;
constexpr size_t NOALLOC_TILES = (size_t)((NOALLOC_MAX_CELLS + 1 + pi::SCAN_TILE - 1) / pi::SCAN_TILE);
constexpr size_t NOALLOC_BYTES = sizeof(pi::Ctrl) + NOALLOC_TILES * sizeof(unsigned long long);
constexpr int NOALLOC_MAX_DEVICES = 64;

void* g_scratch_addr[NOALLOC_MAX_DEVICES];
cudaError_t g_setup_err[NOALLOC_MAX_DEVICES];
std::once_flag g_setup_once[NOALLOC_MAX_DEVICES];

}  // namespace

namespace pi {
void set_last_error_text(const char* text);
}

// Control block followed by the tile descriptors; shared by every call.
static __device__ __align__(256) unsigned char g_scan_scratch[NOALLOC_BYTES];

extern "C" pi_status pi_scan_counts_noalloc(const uint32_t* counts, int64_t C, uint32_t* offsets,
                                            uint32_t* result, pi_stream stream)
{
    char msg[200];
    if (!counts || !offsets || C < 1) return PI_ERR_INVALID_ARG;
    if (C > NOALLOC_MAX_CELLS) {
        std::snprintf(msg, sizeof msg,
                      "pi_scan_counts_noalloc: %lld cells exceed the fixed scratch limit of %lld",
                      (long long)C, (long long)NOALLOC_MAX_CELLS);
        pi::set_last_error_text(msg);
        return PI_ERR_CAPACITY;
    }
    // the scan reads the counts and writes the offsets 16 bytes at a time
    if ((((uintptr_t)counts | (uintptr_t)offsets) & 15u) != 0u || ((uintptr_t)result & 3u) != 0u) {
        pi::set_last_error_text(
            "pi_scan_counts_noalloc: counts and offsets must be 16-byte aligned, result 4-byte aligned");
        return PI_ERR_INVALID_ARG;
    }
    int dev = 0;
    const cudaError_t ge = cudaGetDevice(&dev);
    if (ge != cudaSuccess) {
        std::snprintf(msg, sizeof msg, "pi_scan_counts_noalloc: cudaGetDevice: %s", cudaGetErrorName(ge));
        pi::set_last_error_text(msg);
        return PI_ERR_CUDA;
    }
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        std::snprintf(msg, sizeof msg, "pi_scan_counts_noalloc: device %d is beyond the %d devices it serves", dev,
                      NOALLOC_MAX_DEVICES);
        pi::set_last_error_text(msg);
        return PI_ERR_CAPACITY;
    }
    // once per device, with that device current: the device address of the array
    std::call_once(g_setup_once[dev], [dev] {
        g_setup_err[dev] = cudaGetSymbolAddress(&g_scratch_addr[dev], g_scan_scratch);
    });
    if (g_setup_err[dev] != cudaSuccess || !g_scratch_addr[dev]) {
        // the failed look-up is kept: later calls on this device fail the same way
        std::snprintf(msg, sizeof msg,
                      "pi_scan_counts_noalloc: cudaGetSymbolAddress of the scratch array failed on device %d "
                      "(%s); the failure is kept for this device",
                      dev, cudaGetErrorName(g_setup_err[dev]));
        pi::set_last_error_text(msg);
        return PI_ERR_CUDA;
    }

    cudaStream_t s = (cudaStream_t)stream;
    char* base = (char*)g_scratch_addr[dev];
    pi::Ctrl* ctrl = (pi::Ctrl*)base;
    unsigned long long* status = (unsigned long long*)(base + sizeof(pi::Ctrl));
    const size_t tiles = (size_t)((C + 1 + pi::SCAN_TILE - 1) / pi::SCAN_TILE);
    // the array keeps the previous call's contents: clear the control block
    // and the descriptors this call uses (a cleared descriptor reads as "not
    // ready", so one fixed epoch suffices)
    const size_t words = (sizeof(pi::Ctrl) + tiles * sizeof(unsigned long long)) / 4;
    cudaError_t e = pi::launch_zero((uint32_t*)base, words, nullptr, nullptr, 0, s);
    if (e == cudaSuccess) e = pi::launch_scan(counts, (uint32_t)C, offsets, status, ctrl, 1u, 1000000000ull, 0, s);
    if (e == cudaSuccess && result)
        e = cudaMemcpyAsync(result, &ctrl->max_per_cell, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && result)
        e = cudaMemcpyAsync(result + 1, &ctrl->error, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
        std::snprintf(msg, sizeof msg, "pi_scan_counts_noalloc: launch: %s", cudaGetErrorName(e));
        pi::set_last_error_text(msg);
        return PI_ERR_CUDA;
    }
    return PI_OK;
}
