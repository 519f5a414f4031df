// The static restoration rule (Section 5.2) for one value, shared by the
// restoration kernels (pixel.cu) and the fused row pass (rowfft.cu).
#pragma once

namespace se2n {

// Static restoration. h(t) = max_r scale*Re vol, h(0) = max_r of the lift;
// sigma = (eps h(0) + (1-eps) h(t)) / h(t) where h(t) > guard h(0) and
// h(t) > 0, else the linear blend eps * lift + (1-eps) * psi.
__device__ __forceinline__ float sr_value(float re, float h0, float ht, float lift_r, bool good, float eps,
                                          float guard) {
    if (!good) return re;
    if (ht > guard * h0 && ht > 0.0f) {
        const float sig = (eps * h0 + (1.0f - eps) * ht) / ht;
        return re * sig;
    }
    return eps * lift_r + (1.0f - eps) * re;
}

}  // namespace se2n
