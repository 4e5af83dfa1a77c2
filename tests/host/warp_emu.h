// Host emulation of CUDA thread blocks, for building device code on the CPU
// in the tests.  Every thread of a CTA runs as a host thread (CTAs one after
// another); every warp collective (shuffle, vote, __syncwarp) is a rendezvous
// of the warp's 32 threads at a barrier, __syncthreads one of the whole CTA.
// The code run this way must be warp-uniform (every lane reaches the same
// collectives in the same order), as full-mask collectives require on the
// device too.  Exchanges go through two alternating slot rows, so one barrier
// per collective suffices: a row is written again only two collectives
// later, after every lane has read it.  Storage a CTA shares is declared
// through ABCMB_CTA_SHARED, static here.  Include this header in one
// translation unit only: it defines the emulation's thread-local state.
#pragma once

#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

#include <sched.h>

#define __device__
#define __host__
#define __forceinline__ inline
#define __global__
#define __constant__
#define __shared__
#define __launch_bounds__(...)
#define ABCMB_CTA_SHARED static

struct alignas(16) double2 {
    double x, y;
};
struct alignas(8) float2 {
    float x, y;
};

struct EmuDim3 {
    unsigned x = 0, y = 0, z = 0;
};
extern thread_local EmuDim3 threadIdx, blockIdx, blockDim;

namespace emu {

// generation-counting barrier: spin briefly, then yield (a CTA's threads share
// few cores; under ThreadSanitizer, where every spin is instrumented, yield at
// once); a wait longer than kDeadlineS means lanes disagree about the
// collectives, and the process ends with a message rather than hanging
#if defined(__SANITIZE_THREAD__)
constexpr long kSpins = 0;
#else
constexpr long kSpins = 64;
#endif
struct Barrier {
    explicit Barrier(int n_) : n(n_) {}
    std::atomic<int> count{0}, gen{0};
    const int n;
    void wait()
    {
        constexpr double kDeadlineS = 120.0;
        const int g = gen.load(std::memory_order_acquire);
        if (count.fetch_add(1, std::memory_order_acq_rel) == n - 1) {
            count.store(0, std::memory_order_relaxed);
            gen.fetch_add(1, std::memory_order_release);
            return;
        }
        long spins = 0;
        auto t0 = std::chrono::steady_clock::now();
        while (gen.load(std::memory_order_acquire) == g) {
            if (++spins > kSpins) sched_yield();
            if ((spins & 0xfffff) == 0 &&
                std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > kDeadlineS) {
                std::fprintf(stderr, "warp emulation: lanes never met at a collective\n");
                std::_Exit(3);
            }
        }
    }
};

struct Warp {
    Barrier bar{32};
    uint64_t slot[2][32];
};

struct Cta {
    explicit Cta(int n) : bar(n) {}
    Barrier bar;
};

extern thread_local Warp *warp;
extern thread_local Cta *cta;
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

// run one CTA of n threads (a multiple of 32) as host threads: body() is the
// kernel body, called with threadIdx, blockIdx, blockDim and the warp set up
template <class F>
void run_cta(unsigned bx, unsigned by, int n, F &&body);

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
inline int __reduce_max_sync(unsigned, int v)
{
    uint64_t *row = emu::warp->slot[emu::parity];
    emu::parity ^= 1;
    row[emu::lane] = (uint64_t)(uint32_t)v;
    emu::warp->bar.wait();
    int m = (int)(uint32_t)row[0];
    for (int i = 1; i < 32; i++) m = (int)(uint32_t)row[i] > m ? (int)(uint32_t)row[i] : m;
    return m;
}
inline void __syncwarp(unsigned = 0xffffffffu) { emu::warp->bar.wait(); }
inline void __syncthreads() { emu::cta->bar.wait(); }

inline double atomicAdd(double *p, double v)
{
    double old, want;
    __atomic_load(p, &old, __ATOMIC_RELAXED);
    do want = old + v;
    while (!__atomic_compare_exchange(p, &old, &want, true, __ATOMIC_ACQ_REL, __ATOMIC_RELAXED));
    return old;
}

inline int __popc(unsigned x) { return __builtin_popcount(x); }
inline int __double2hiint(double d) { return (int)(uint32_t)(emu::bits_of(d) >> 32); }
inline double __hiloint2double(int hi, int lo)
{
    return emu::from_bits<double>(((uint64_t)(uint32_t)hi << 32) | (uint32_t)lo);
}
inline float __powf(float x, float y) { return powf(x, y); }
// single-precision operations rounded once each (the harnesses build with
// floating-point contraction off)
inline float __fadd_rn(float a, float b) { return a + b; }
inline float __fsub_rn(float a, float b) { return a - b; }
inline float __fmul_rn(float a, float b) { return a * b; }
inline int max(int a, int b) { return a > b ? a : b; }
inline int min(int a, int b) { return a < b ? a : b; }

thread_local EmuDim3 threadIdx, blockIdx, blockDim;
namespace emu {
thread_local Warp *warp = nullptr;
thread_local Cta *cta = nullptr;
thread_local int lane = 0;
thread_local int parity = 0;

template <class F>
void run_cta(unsigned bx, unsigned by, int n, F &&body)
{
    Cta c(n);
    std::vector<Warp> warps(n / 32);
    std::vector<std::thread> th;
    th.reserve(n);
    for (int t = 0; t < n; t++)
        th.emplace_back([&, t] {
            warp = &warps[t / 32];
            cta = &c;
            lane = t & 31;
            parity = 0;
            threadIdx.x = t;
            blockIdx.x = bx;
            blockIdx.y = by;
            blockDim.x = n;
            body();
        });
    for (auto &x : th) x.join();
}
} // namespace emu
