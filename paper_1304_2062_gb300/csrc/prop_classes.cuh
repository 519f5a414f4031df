// Classes of frequencies that share one S-step propagator (see propagator.cu):
// the coefficients of frequency (k, l) depend on it only through
// wx = sin(2 pi l / W) and wy = sin(2 pi k / H).
#pragma once

namespace se2n {

// Rows k and (H/2 - k) mod H have bitwise the same coefficients:
// sin_2pi_frac folds 2 pi k / H with integer arithmetic to the same argument
// of sinpif for both (up to the sign of a zero, which the square removes).
// The pairs are enumerated once each: k in [0, H/4] (partner H/2 - k) and
// k in [H/2 + 1, 3H/4] (partner 3H/2 - k); k = H/4 and 3H/4 are their own
// partners. H is even. Columns of the full spectrum are paired this way.
__host__ __device__ __forceinline__ int pair_rows(int H) { return H / 4 + 1 + (3 * H) / 4 - H / 2; }
__device__ __forceinline__ void pair_row(int s, int H, int &k, int &kb) {
    const int lo = H / 4 + 1;
    k = (s < lo) ? s : H / 2 + 1 + (s - lo);
    kb = (k <= H / 2) ? H / 2 - k : 3 * H / 2 - k;
}

// Row slot s in [0, H/4] (H even): rows s and H/2 - s with wy = sin(2 pi s / H)
// (the coefficients the propagator is built for) and rows H/2 + s and
// (H - s) mod H with -wy (taken with the angles reversed). Each row of the
// plane is in exactly one slot: s = 0 holds rows 0 and H/2 only, and s = H/4
// rows H/4 and 3H/4 only.
__host__ __device__ __forceinline__ int row_slots(int H) { return H / 4 + 1; }
__host__ __device__ __forceinline__ void slot_rows(int s, int H, int (&k)[4], bool (&on)[4]) {
    k[0] = s;
    k[1] = H / 2 - s;
    k[2] = H / 2 + s;
    k[3] = (H - s) % H;
    const bool quarter = 4 * s == H;
    on[0] = true;
    on[1] = !quarter;
    on[2] = s != 0;
    on[3] = s != 0 && !quarter;
}

// The slots of a system of NE = N - 2 angles (30 in 32) in the row and
// column passes, whose kernels are written for N: angle r < NE/2 at slot r,
// NE/2 at slot N/2, r > NE/2 at slot r + 2; slots NE/2 and N/2 + 1 stay empty
// (zero in every plane and in every propagator's rows and columns). Angle
// reversal modulo NE is then slot reversal modulo N, which the column pass
// does. angle_of_slot gives NE, NE + 1 for the two empty slots; NE = N is the
// identity.
template <int N, int NE>
__host__ __device__ constexpr int slot_of_angle(int r) {
    return NE == N ? r : (r < NE / 2 ? r : (r == NE / 2 ? N / 2 : r + 2));
}
template <int N, int NE>
__host__ __device__ constexpr int angle_of_slot(int s) {
    return NE == N ? s
                   : (s < NE / 2 ? s
                                 : (s == NE / 2 ? NE : (s == N / 2 ? NE / 2 : (s == N / 2 + 1 ? NE + 1 : s - 2))));
}
static_assert(angle_of_slot<32, 30>(slot_of_angle<32, 30>(15)) == 15 &&
                  angle_of_slot<32, 30>(slot_of_angle<32, 30>(29)) == 29 && slot_of_angle<32, 30>(29) == 31 &&
                  (32 - slot_of_angle<32, 30>(1)) % 32 == slot_of_angle<32, 30>(29),
              "the slots of 30 angles in 32");

// Column slot of column l of the Hermitian half (l in [0, W/2]): columns l
// and W/2 - l share slot min(l, W/2 - l) in [0, W/4].
__host__ __device__ __forceinline__ int half_col_slot(int l, int W) { return l <= W / 4 ? l : W / 2 - l; }

}  // namespace se2n
