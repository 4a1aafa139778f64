// lb_warp.cuh -- warp-tile helpers shared by the warp-tiled kernels (the merge-path product
// and the CSR-order backward pass): tile geometry, the padded per-warp value buffer, 256-bit
// streaming loads and stores, and slot masks.
#pragma once

#include <type_traits>

#include "lb_internal.cuh"

namespace lb {

// Warp tile geometry.  A tile's first nonzero sits `lead` (0..7) slots past a 32-byte
// boundary of the index array, so every lane's IPT slots start 32-byte aligned and a tile
// holds at most 32 * IPT - 8 work items.
template <int IPT>
struct WarpTile {
    static_assert(IPT == 8 || IPT == 16, "8 or 16 slots per lane");
    static constexpr int SLOTS = 32 * IPT;
    static constexpr int ITEMS = SLOTS - 8;
    // Per warp in shared memory: the tile's scanned slot values (4 floats of padding after
    // every 32 keep the lanes' 128-bit accesses free of bank conflicts), then one row-start
    // flag byte per slot.
    static constexpr int VALS = SLOTS + SLOTS / 8;
    static constexpr int BYTES = VALS * 4 + SLOTS;
};

// Index of slot j in the padded value buffer.
__device__ __forceinline__ int ppad(int j) { return j + ((j >> 5) << 2); }

// Streaming loads: 256 or 128 bits per lane, L1 bypassed, L2 evict-first.
__device__ __forceinline__ void ld_stream8(const void *p, uint64_t pol, uint32_t (&r)[8]) {
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8], %9;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "l"(p), "l"(pol));
}

__device__ __forceinline__ void ld_stream4(const void *p, uint64_t pol, uint32_t (&r)[4]) {
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.b32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "l"(p), "l"(pol));
}

__device__ __forceinline__ void st_stream8(void *p, uint64_t pol, const float *v) {
    asm volatile("st.global.L1::no_allocate.L2::cache_hint.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8}, %9;" ::"l"(p),
                 "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "l"(pol)
                 : "memory");
}

// Lane mask of this lane's slots that hold the tile's nonzeros: slot q holds element e0 + q.
template <int IPT>
__device__ __forceinline__ uint32_t slot_mask(int e0, int k0, int k1) {
    const int lo = min(max(k0 - e0, 0), IPT);  // slots [lo, hi) lie in [k0, k1)
    const int hi = min(max(k1 - e0, 0), IPT);
    return ((1u << hi) - 1u) & ~((1u << lo) - 1u);
}

// A 16-bit value's bits widened to FP32 (BF16: shift into the high half; FP16: convert).
template <typename V>
__device__ __forceinline__ float half_bits_to_f32(uint32_t bits) {
    if constexpr (std::is_same<V, __nv_bfloat16>::value)
        return __uint_as_float(bits << 16);
    else
        return __half2float(__ushort_as_half(static_cast<unsigned short>(bits)));
}

}  // namespace lb
