// Packed FP32x2 arithmetic (sm_100 and later): two IEEE FP32 operations per
// instruction, each lane rounded exactly as the scalar _rn operation.  Unlike
// the scalar _rn intrinsics, a packed multiply feeding a packed add may be
// fused into one packed fma by the compiler (measured on sm_103a), so code
// that must reproduce a fixed rounding sequence writes its fmas explicitly.
#pragma once

namespace dn {
namespace {

struct f2 {
    unsigned long long v;
};
__device__ __forceinline__ f2 f2_pack(float lo, float hi)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2 a, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
}
__device__ __forceinline__ float f2_lo(f2 a)
{
    return __uint_as_float((unsigned)(a.v & 0xFFFFFFFFull));
}
__device__ __forceinline__ float f2_hi(f2 a)
{
    return __uint_as_float((unsigned)(a.v >> 32));
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b)
{
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b)
{
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b)
{
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c)
{
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
    return r;
}

// (a - b)^2 per lane (the compiler may fuse the product into a following
// packed add).
__device__ __forceinline__ f2 f2_sqd(f2 a, f2 b)
{
    const f2 e = f2_sub(a, b);
    return f2_mul(e, e);
}

}  // namespace
}  // namespace dn
