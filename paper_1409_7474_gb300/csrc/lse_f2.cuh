// lse_f2.cuh -- packed pairs of FP32 values for the step kernels.
#pragma once

// Two FP32 values in one 64-bit register pair.  Blackwell's packed FP32
// instructions (add / mul / fma .rn.f32x2) round each element exactly as the
// scalar instruction does, in one instruction for the pair.
struct f2 {
    unsigned long long r;
};

__device__ __forceinline__ f2 f2_pack(float a, float b)
{
    f2 o;
    asm("mov.b64 %0, {%1, %2};" : "=l"(o.r) : "f"(a), "f"(b));
    return o;
}

__device__ __forceinline__ void f2_unpack(f2 v, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v.r));
}

__device__ __forceinline__ f2 f2_add(f2 a, f2 b)
{
    f2 o;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(o.r) : "l"(a.r), "l"(b.r));
    return o;
}

__device__ __forceinline__ f2 f2_sub(f2 a, f2 b)
{
    f2 o;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(o.r) : "l"(a.r), "l"(b.r));
    return o;
}

__device__ __forceinline__ f2 f2_mul(f2 a, f2 b)
{
    f2 o;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(o.r) : "l"(a.r), "l"(b.r));
    return o;
}

__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c)
{
    f2 o;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(o.r) : "l"(a.r), "l"(b.r), "l"(c.r));
    return o;
}
