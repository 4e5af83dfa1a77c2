// Host emulation of one CUDA warp, for building warp-level device code on
// the CPU in the tests.  The 32 lanes run as host threads; every warp
// collective (shuffle, vote, __syncwarp) is a rendezvous of all 32 at a
// barrier.  The code run this way must be warp-uniform (every lane reaches
// the same collectives in the same order), as full-mask collectives require
// on the device too.  Exchanges go through two alternating slot rows, so one
// barrier per collective suffices: a row is written again only two
// collectives later, after every lane has read it.
#pragma once

#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <sched.h>

#define __device__
#define __forceinline__ inline
#define __global__
#define __constant__
#define __shared__
#define __launch_bounds__(...)

struct EmuDim3 {
    unsigned x = 0, y = 0, z = 0;
};
extern thread_local EmuDim3 threadIdx, blockIdx, blockDim;

namespace emu {

// sense-counting barrier: spin briefly, then yield (32 threads share few
// cores); a wait longer than kDeadlineS means lanes disagree about the
// collectives, and the process ends with a message rather than hanging
struct Barrier {
    std::atomic<int> count{0}, gen{0};
    void wait()
    {
        constexpr double kDeadlineS = 120.0;
        const int g = gen.load(std::memory_order_acquire);
        if (count.fetch_add(1, std::memory_order_acq_rel) == 31) {
            count.store(0, std::memory_order_relaxed);
            gen.fetch_add(1, std::memory_order_release);
            return;
        }
        long spins = 0;
        auto t0 = std::chrono::steady_clock::now();
        while (gen.load(std::memory_order_acquire) == g) {
            if (++spins > 64) sched_yield();
            if ((spins & 0xfffff) == 0 &&
                std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > kDeadlineS) {
                std::fprintf(stderr, "warp emulation: lanes never met at a collective\n");
                std::_Exit(3);
            }
        }
    }
};

struct Warp {
    Barrier bar;
    uint64_t slot[2][32];
};

extern thread_local Warp *warp;
extern thread_local int lane;
extern thread_local int parity;

template <class T>
inline uint64_t bits_of(T v)
{
    static_assert(sizeof(T) <= 8, "one register");
    uint64_t b = 0;
    std::memcpy(&b, &v, sizeof(T));
    return b;
}

template <class T>
inline T from_bits(uint64_t b)
{
    T v;
    std::memcpy(&v, &b, sizeof(T));
    return v;
}

// every lane posts v, then reads lane src's post
template <class T>
inline T exchange(T v, int src)
{
    uint64_t *row = warp->slot[parity];
    parity ^= 1;
    row[lane] = bits_of(v);
    warp->bar.wait();
    return from_bits<T>(row[src]);
}

inline unsigned ballot(bool p)
{
    uint64_t *row = warp->slot[parity];
    parity ^= 1;
    row[lane] = p ? 1u : 0u;
    warp->bar.wait();
    unsigned m = 0;
    for (int i = 0; i < 32; i++) m |= (unsigned)row[i] << i;
    return m;
}

} // namespace emu

template <class T>
inline T __shfl_sync(unsigned, T v, int src, int width = 32)
{
    return emu::exchange(v, (emu::lane & ~(width - 1)) + (src & (width - 1)));
}

template <class T>
inline T __shfl_up_sync(unsigned, T v, unsigned d, int width = 32)
{
    const int w = emu::lane & (width - 1);
    return emu::exchange(v, w >= (int)d ? emu::lane - (int)d : emu::lane);
}

template <class T>
inline T __shfl_down_sync(unsigned, T v, unsigned d, int width = 32)
{
    const int w = emu::lane & (width - 1);
    return emu::exchange(v, w + (int)d < width ? emu::lane + (int)d : emu::lane);
}

template <class T>
inline T __shfl_xor_sync(unsigned, T v, int m, int width = 32)
{
    const int src = emu::lane ^ m;
    return emu::exchange(v, (src & ~(width - 1)) == (emu::lane & ~(width - 1)) ? src : emu::lane);
}

inline unsigned __ballot_sync(unsigned, int p) { return emu::ballot(p != 0); }
inline int __any_sync(unsigned, int p) { return emu::ballot(p != 0) != 0u; }
inline int __all_sync(unsigned, int p) { return emu::ballot(p != 0) == 0xffffffffu; }
inline void __syncwarp(unsigned = 0xffffffffu) { emu::warp->bar.wait(); }
inline void __syncthreads() { emu::warp->bar.wait(); }

inline int __popc(unsigned x) { return __builtin_popcount(x); }
inline int __double2hiint(double d) { return (int)(uint32_t)(emu::bits_of(d) >> 32); }
inline double __hiloint2double(int hi, int lo)
{
    return emu::from_bits<double>(((uint64_t)(uint32_t)hi << 32) | (uint32_t)lo);
}
inline float __powf(float x, float y) { return powf(x, y); }
inline int max(int a, int b) { return a > b ? a : b; }
inline int min(int a, int b) { return a < b ? a : b; }
