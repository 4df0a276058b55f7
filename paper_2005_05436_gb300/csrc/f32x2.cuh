// Two FP32 lanes in one 64-bit register, operated on by the paired FP32
// instructions of sm_100-class GPUs (add/sub/mul/fma .f32x2 in PTX). Each lane
// is rounded exactly as the scalar FP32 instruction would round it (.rn), so a
// kernel written on F2 gives, lane by lane, the results of the same scalar
// code, with half the instructions issued. Arithmetic operators are provided
// so that templated element code (walsh.cuh) runs on F2 unchanged.
#pragma once

#include <cstdint>

namespace topo {

struct F2 {
    unsigned long long v;
    F2() = default;
    __device__ __forceinline__ explicit F2(float a) { v = pack(a, a); }
    __device__ __forceinline__ explicit F2(int a) { v = pack((float)a, (float)a); }
    __device__ __forceinline__ static unsigned long long pack(float lo, float hi) {
        unsigned long long r;
        asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
        return r;
    }
    __device__ __forceinline__ static F2 make(float lo, float hi) {
        F2 r;
        r.v = pack(lo, hi);
        return r;
    }
    __device__ __forceinline__ float lo() const {
        float a;
        asm("{\n\t.reg .b32 t;\n\tmov.b64 {%0, t}, %1;\n\t}" : "=f"(a) : "l"(v));
        return a;
    }
    __device__ __forceinline__ float hi() const {
        float b;
        asm("{\n\t.reg .b32 t;\n\tmov.b64 {t, %0}, %1;\n\t}" : "=f"(b) : "l"(v));
        return b;
    }
};

__device__ __forceinline__ F2 operator+(F2 a, F2 b) {
    F2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 operator-(F2 a, F2 b) {
    F2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ F2 operator*(F2 a, F2 b) {
    F2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
// Negation flips both sign bits (exact, like the scalar negation).
__device__ __forceinline__ F2 operator-(F2 a) {
    F2 r;
    r.v = a.v ^ 0x8000000080000000ull;
    return r;
}
// a * b + c with one rounding per lane.
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) {
    F2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}

}  // namespace topo
