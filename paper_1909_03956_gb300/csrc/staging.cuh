// staging.cuh -- per-CTA streaming of a read-only record list through shared
// memory with bulk (TMA, non-tensor, non-multicast) copies and mbarriers.
//
// Every thread of the CTA walks the same records in the same order (each
// thread owns a different visibility), so a record is read from shared
// memory as a broadcast. Two buffers of `chunk` records alternate: while the
// CTA works on one, the next chunk is in flight into the other. A list that
// fits in the two buffers is loaded once and stays resident for every tile
// the CTA processes.
#pragma once

#include <type_traits>

#include "wt_internal.cuh"

namespace wt {

template <class Rec>
struct Stager {
    const Rec* recs;      // global, 16-byte aligned, readable up to a 16-byte multiple
    int64_t count;        // records in the list
    Rec* buf;             // shared, 2 * chunk records
    uint64_t* bars;       // shared, 2 mbarriers
    int chunk;            // records per buffer (even, so chunk * sizeof(Rec) % 16 == 0)
    uint32_t phase0, phase1;  // expected parity per buffer
    bool busy0, busy1;    // a copy into buffer 0 / 1 has been issued and not yet waited for
    bool resident;        // whole list fits in the two buffers
    bool loaded;          // resident list already in shared memory

    __device__ int64_t nchunks() const { return (count + chunk - 1) / chunk; }

    __device__ void issue(int64_t c, int b)
    {
        const int64_t first = c * chunk;
        const int64_t n = (count - first < chunk) ? (count - first) : chunk;
        const uint32_t bytes = static_cast<uint32_t>(((n * static_cast<int64_t>(sizeof(Rec))) + 15) & ~int64_t(15));
        mbar_arrive_expect_tx(&bars[b], bytes);
        bulk_copy_g2s(buf + static_cast<int64_t>(b) * chunk, recs + first, bytes, &bars[b]);
    }

    // Called by all threads once, after the barriers are initialised.
    __device__ void init_state()
    {
        phase0 = phase1 = 0;
        busy0 = busy1 = false;
        resident = nchunks() <= 2;
        loaded = false;
    }

    // After a wait ran out: one more bounded wait on every buffer whose copy
    // is still outstanding, so that the CTA does not exit while a bulk copy
    // may still write into its shared memory. Called by every thread (the
    // busy flags are uniform across the CTA). If a copy still has not
    // arrived, the CTA leaves anyway; the caller has recorded WT_ERR_TIMEOUT
    // and the device's later results are not to be trusted.
    __device__ void drain()
    {
        if (busy0) mbar_wait_parity(&bars[0], phase0);
        if (busy1) mbar_wait_parity(&bars[1], phase1);
    }

    // Point the stager at another record list (same chunking). Call only
    // when no copy is in flight (after a completed sweep) and after a CTA
    // barrier, so that no thread still reads the buffers.
    __device__ void retarget(const Rec* r, int64_t n)
    {
        recs = r;
        count = n;
        resident = nchunks() <= 2;
        loaded = false;
    }

    // Run body(rec) for every record, in order. Returns false (uniformly
    // across the CTA) if a copy did not arrive within the spin limit.
    template <class Body>
    __device__ bool sweep(Body& body)
    {
        const int64_t nc = nchunks();
        if (nc == 0) return true;
        const bool need_load = !(resident && loaded);
        if (need_load && threadIdx.x == 0) {
            issue(0, 0);
            if (nc > 1) issue(1, 1);
        }
        if (need_load) {
            busy0 = true;
            busy1 = nc > 1;
        }
        for (int64_t c = 0; c < nc; ++c) {
            const int b = static_cast<int>(c & 1);
            if (need_load) {
                const bool ok = mbar_wait_parity(&bars[b], b ? phase1 : phase0);
                if (!__syncthreads_and(ok ? 1 : 0)) {
                    drain();
                    return false;
                }
                if (b) {
                    phase1 ^= 1u;
                    busy1 = false;
                } else {
                    phase0 ^= 1u;
                    busy0 = false;
                }
            }
            const int64_t first = c * chunk;
            const int n = static_cast<int>((count - first < chunk) ? (count - first) : chunk);
            const Rec* cb = buf + static_cast<int64_t>(b) * chunk;
            // four records per trip: a quarter of the loop overhead per record
            // (measured: the mixed predictors 8-9 % faster than one per trip,
            // 3 % faster than two; eight gains 1 % more)
#pragma unroll 4
            for (int r = 0; r < n; ++r) body(cb[r]);
            if (!resident) {
                __syncthreads();                           // buffer b fully consumed
                if (threadIdx.x == 0 && c + 2 < nc) issue(c + 2, b);
                if (c + 2 < nc) {
                    if (b) busy1 = true;
                    else busy0 = true;
                }
            }
        }
        if (resident) loaded = true;
        return true;
    }

    // As sweep, but the body sees the chunk, the position and the chunk's
    // record count (body.at(chunk, r, n)), so that it may handle a record
    // together with its neighbours: a body whose at() returns the number of
    // records it took (at least 1) advances by it.
    template <class Body>
    __device__ bool sweep_at(Body& body)
    {
        const int64_t nc = nchunks();
        if (nc == 0) return true;
        const bool need_load = !(resident && loaded);
        if (need_load && threadIdx.x == 0) {
            issue(0, 0);
            if (nc > 1) issue(1, 1);
        }
        if (need_load) {
            busy0 = true;
            busy1 = nc > 1;
        }
        for (int64_t c = 0; c < nc; ++c) {
            const int b = static_cast<int>(c & 1);
            if (need_load) {
                const bool ok = mbar_wait_parity(&bars[b], b ? phase1 : phase0);
                if (!__syncthreads_and(ok ? 1 : 0)) {
                    drain();
                    return false;
                }
                if (b) {
                    phase1 ^= 1u;
                    busy1 = false;
                } else {
                    phase0 ^= 1u;
                    busy0 = false;
                }
            }
            const int64_t first = c * chunk;
            const int n = static_cast<int>((count - first < chunk) ? (count - first) : chunk);
            const Rec* cb = buf + static_cast<int64_t>(b) * chunk;
            if constexpr (std::is_void_v<decltype(body.at(cb, 0, n))>) {
                // four records per trip (measured against two: 2 % faster on
                // the blob workloads, 4-6 % slower on deep trees of isolated
                // components, whose records are mostly internal nodes)
#pragma unroll 4
                for (int r = 0; r < n; ++r) body.at(cb, r, n);
            } else {
                // the body takes one or more records per step
                for (int r = 0; r < n;) r += body.at(cb, r, n);
            }
            if (!resident) {
                __syncthreads();
                if (threadIdx.x == 0 && c + 2 < nc) issue(c + 2, b);
                if (c + 2 < nc) {
                    if (b) busy1 = true;
                    else busy0 = true;
                }
            }
        }
        if (resident) loaded = true;
        return true;
    }
};

// Shared-memory layout helper: bytes for the two record buffers plus the two
// mbarriers, rounded to 16.
template <class Rec>
__host__ __device__ constexpr int64_t stager_bytes(int chunk)
{
    return ((2 * static_cast<int64_t>(chunk) * static_cast<int64_t>(sizeof(Rec)) + 16 + 15) / 16) * 16;
}

template <class Rec>
__device__ __forceinline__ void stager_setup(Stager<Rec>& st, unsigned char* smem, const Rec* recs, int64_t count,
                                             int chunk)
{
    st.recs = recs;
    st.count = count;
    st.chunk = chunk;
    st.buf = reinterpret_cast<Rec*>(smem);
    st.bars = reinterpret_cast<uint64_t*>(smem + 2 * static_cast<int64_t>(chunk) * sizeof(Rec));
    if (threadIdx.x == 0) {
        mbar_init(&st.bars[0], 1);
        mbar_init(&st.bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    st.init_state();
}

}  // namespace wt
