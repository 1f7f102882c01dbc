// Packed two-lane FP32 arithmetic (sm_100 and later): one instruction
// applies the same operation to the x and y lanes of float2 operands, each
// lane rounded exactly as the scalar operation would be.  Sums, products and
// fused multiply-adds come from the CUDA intrinsics (__fadd2_rn, __fmul2_rn,
// __ffma2_rn); the difference has no intrinsic, so it is written here.
#pragma once

#include <cuda_runtime.h>

namespace fdkod {

// a - b in both lanes, round to nearest
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\t"
        "mov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

}  // namespace fdkod
