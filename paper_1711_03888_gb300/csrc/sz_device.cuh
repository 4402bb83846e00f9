// sz_device.cuh -- device helpers shared by the GB300 kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "sz_internal.h"

namespace szg {

__host__ __device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a > b ? a : b; }
__host__ __device__ __forceinline__ uint32_t umin32(uint32_t a, uint32_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ uint32_t umax32(uint32_t a, uint32_t b) { return a > b ? a : b; }

// ---------------------------------------------------------------------------
// Order-preserving float <-> u32 keys (for min/max with integer atomics)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t float_key(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_float(uint32_t k) {
    uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(u);
}
__device__ __forceinline__ bool finite_f(float x) {
    return (__float_as_uint(x) & 0x7f800000u) != 0x7f800000u;
}

// ---------------------------------------------------------------------------
// Sec. III: error bound and lattice step from the value range.
// D = largest float <= 2*eb_abs (clamped to FLT_MAX); the verbatim test
// |x - RN32(qD)| > eb_abs is exact in float form as |x - xr| > RD32(eb_abs).
// ---------------------------------------------------------------------------
__device__ __forceinline__ LatticeParams make_params(double eb_abs) {
    LatticeParams P;
    P.eb_abs = eb_abs;
    double two = __dmul_rn(2.0, eb_abs);
    float D = (two >= 3.4028234663852886e38) ? 3.4028234663852886e38f : __double2float_rz(two);
    P.D = D;
    P.raw = (D == 0.0f);
    P.fast = (D >= 7.888609052210118e-31f /*2^-100*/ && D <= 1.2676506002282294e30f /*2^100*/);
    P.inv = P.raw ? 0.0f : __fdiv_rn(1.0f, D);
    // D*(1/2 -+ 2^-20) is exact in binary64 (24 + 20 bits); round outward/inward to float
    P.thr_lo = __double2float_rd(__dmul_rn((double)D, 0.5 - 9.5367431640625e-07));
    P.thr_hi = __double2float_ru(__dmul_rn((double)D, 0.5 + 9.5367431640625e-07));
    P.ebf = __double2float_rd(eb_abs);
    return P;
}

__device__ __forceinline__ double range_eb_abs(double eb, int kind, uint32_t min_key, uint32_t max_key,
                                               uint32_t any) {
    if (kind == 0) return eb;
    if (!any) return 0.0;
    double R = __dsub_rn((double)key_float(max_key), (double)key_float(min_key));
    return __dmul_rn(eb, R);
}

// ---------------------------------------------------------------------------
// Value -> lattice (a2) and the verbatim decision.
// Definition: t = RN64(x / D); q = RNE(t) if x finite and |t| < 2^53, else
// q = 0 (verbatim); verbatim also when |x - RN32(RN64(q*D))| > eb_abs.
// Fast path (pure FP32, exact): candidate qc = rint(x*inv), residual
// r = RN32(x - qc*D) by one fma.  |r| <= thr_lo proves |x/D - qc| < 1/2 -
// 2^-21, so RNE(RN64(x/D)) = qc.  Then q*D (<= 47 bits) is exact in binary64,
// RN32(RN64(qD)) = RN32(qD) = one fmul, and x - xr is exact (Sterbenz), so
// the float test |x - xr| > RD32(eb_abs) equals the binary64 test.
// Near-ties (thr_lo < |r| < thr_hi, probability ~2^-19) and out-of-range
// candidates fall back to the binary64 definition.
// ---------------------------------------------------------------------------
struct LatticeOut {
    long long q;
    int verb;
};

static __device__ __noinline__ LatticeOut lattice_slow(float x, double eb_abs, float D, int raw) {
    LatticeOut o;
    if (!finite_f(x) || raw) { o.q = 0; o.verb = 1; return o; }
    double t = __ddiv_rn((double)x, (double)D);
    if (!(fabs(t) < 9007199254740992.0)) { o.q = 0; o.verb = 1; return o; }
    long long k = __double2ll_rn(t);
    float xr = __double2float_rn(__dmul_rn((double)k, (double)D));
    o.q = k;
    o.verb = fabs(__dsub_rn((double)x, (double)xr)) > eb_abs;
    return o;
}

__device__ __forceinline__ void lattice_q(float x, const LatticeParams& P, long long& q, bool& verb) {
    float t = x * P.inv;
    if (P.fast && fabsf(t) < 4194304.0f /*2^22*/) {   // NaN/Inf fail this test
        float qc = rintf(t);
        float r = fmaf(-qc, P.D, x);
        float ar = fabsf(r);
        bool ok = ar <= P.thr_lo;
        if (!ok && ar >= P.thr_hi) {
            qc += (r > 0.0f) ? 1.0f : -1.0f;
            r = fmaf(-qc, P.D, x);
            ok = fabsf(r) <= P.thr_lo;
        }
        if (ok) {
            float xr = __fmul_rn(qc, P.D);
            q = (long long)(int)qc;
            verb = fabsf(__fsub_rn(x, xr)) > P.ebf;
            return;
        }
    }
    LatticeOut o = lattice_slow(x, P.eb_abs, P.D, P.raw);
    q = o.q;
    verb = o.verb != 0;
}

// Lattice -> value (a11): RN32(RN64(q*D)); one fmul while |q| <= 2^24.
__device__ __forceinline__ float recon_f(long long q, float D) {
    if (q >= -16777216LL && q <= 16777216LL) return __fmul_rn((float)(int)q, D);
    return __double2float_rn(__dmul_rn((double)q, (double)D));
}

// LV prediction + linear-scaling quantization (a3): code = delta + 32768 for
// |delta| <= 32767 and not verbatim; 0 (escape) otherwise.
__device__ __forceinline__ uint32_t make_code(long long q, long long qprev, bool verb) {
    long long d = q - qprev;
    return (!verb && d >= -(kRadius - 1) && d <= (kRadius - 1)) ? (uint32_t)(d + kRadius) : 0u;
}

// ---------------------------------------------------------------------------
// Shared-memory staging layout of a chunk: element e lives at
//   (e & ~31) | (((e >> 2) & 7) ^ ((e / G) & 7)) << 2 | (e & 3)
// i.e. the 16-byte groups of each 128-byte line are XOR-swizzled by the
// sub-stream index.  Coalesced float4 copies (lane l -> elements 4l..4l+3)
// and per-sub-stream float4 walks (thread k -> elements kG+4m..) are then
// both free of bank conflicts.  Requires G a multiple of 32.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t swz(uint32_t e, uint32_t gshift) {
    return (e & ~31u) | ((((e >> 2) & 7u) ^ ((e >> gshift) & 7u)) << 2) | (e & 3u);
}

// ---------------------------------------------------------------------------
// Status-word access for the decoupled look-back.  A chunk's status word holds
// its flag and its value in one 64-bit word, and no other data is handed over
// through it, so relaxed device-scope accesses suffice: a release store would
// make the publishing thread wait for its earlier global writes first.
// Measured on GB300 (six 2^27-element arrays, batched encode): acquire loads
// with release stores 2.60 ms, relaxed loads 2.51 ms, both relaxed 2.23 ms.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void st_status(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_status(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Decoupled look-back over the chunks before chunk c, by one full warp.
// status[j] holds a 2-bit flag and a 62-bit value: AGG (chunk j's own word
// count), INC (the words of chunks 0 .. j) or ERR (chunk j gave up).  Lane l
// reads chunk j - l, 32 predecessors per step, and the warp sums back to the
// nearest INC.  A word still unpublished is polled at most spin_limit times
// (with a short sleep between polls); after that, or on an ERR, the warp
// returns false.  On success every lane gets the exclusive prefix in *excl.
constexpr unsigned long long kLbAgg = 1ull << 62, kLbInc = 2ull << 62, kLbErr = 3ull << 62;
constexpr unsigned long long kLbValue = (1ull << 62) - 1;

__device__ __forceinline__ bool lookback_prefix(const unsigned long long* status, uint64_t c, uint32_t spin_limit,
                                                unsigned long long* excl) {
    const int lane = threadIdx.x & 31;
    unsigned long long sum = 0;
    long long j = (long long)c - 1;
    while (j >= 0) {
        const long long pos = j - lane;
        unsigned long long s = kLbInc;                 // before chunk 0: an empty prefix
        if (pos >= 0) {
            uint32_t spins = 0;
            s = ld_status(&status[pos]);
            while ((s & ~kLbValue) == 0ull && spins < spin_limit) {
                __nanosleep(64);
                s = ld_status(&status[pos]);
                ++spins;
            }
        }
        const unsigned long long f = s & ~kLbValue;
        if (__any_sync(0xffffffffu, f == 0ull || f == kLbErr)) return false;
        const uint32_t inc = __ballot_sync(0xffffffffu, f == kLbInc);
        const int lim = inc ? (__ffs(inc) - 1) : 31;  // lanes 0 .. lim contribute
        unsigned long long v = (lane <= lim) ? (s & kLbValue) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        sum += v;
        if (inc) break;
        j -= 32;
    }
    *excl = sum;
    return true;
}

// ---------------------------------------------------------------------------
// Scans
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Exclusive block scan for blockDim.x == NT (multiple of 32, <= 1024).
// `ws` must hold NT/32 + 1 elements of T.  Returns the exclusive prefix; the
// block total is in *total.  Contains __syncthreads().
template <int NT, typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* ws, T* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T inc = warp_inclusive_scan(v);
    if (lane == 31) ws[w] = inc;
    __syncthreads();
    if (w == 0) {
        T s = (lane < NT / 32) ? ws[lane] : T(0);
        T si = warp_inclusive_scan(s);
        if (lane < NT / 32) ws[lane] = si - s;
        if (lane == NT / 32 - 1) ws[NT / 32] = si;
    }
    __syncthreads();
    T r = ws[w] + inc - v;
    *total = ws[NT / 32];
    __syncthreads();
    return r;
}

template <typename T>
__device__ __forceinline__ T warp_reduce_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void raise_err(uint32_t* err, uint32_t bits) { atomicOr(err, bits); }

__device__ __forceinline__ void st_u64_unaligned(uint8_t* p, uint64_t v) {
    for (int k = 0; k < 8; ++k) p[k] = (uint8_t)(v >> (8 * k));
}

}  // namespace szg
