// Complex butterflies on the packed float32x2 instructions: (re, im) pairs are
// one 64-bit operand, so a complex add or subtract is one instruction instead
// of two, rounded per element exactly as two float32 operations.
#pragma once

#include <stdint.h>

namespace ptdr {

// (a, b) <- (a + b, a - b).
__device__ __forceinline__ void bfly2(float2& a, float2& b)
{
    uint64_t x, y, s, d;
    asm("mov.b64 %0, {%1,%2};" : "=l"(x) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1,%2};" : "=l"(y) : "f"(b.x), "f"(b.y));
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(s) : "l"(x), "l"(y));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(x), "l"(y));
    asm("mov.b64 {%0,%1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(s));
    asm("mov.b64 {%0,%1}, %2;" : "=f"(b.x), "=f"(b.y) : "l"(d));
}

} // namespace ptdr
