// Host-side packing of an on-chip op's coefficients (shared by the
// interpreted and the compiled fused kernels).
//
// complex64: a GEN2 (4x4) op has one set of 16 (re, re), (im, im), (-im, -im)
// triples, row-major. Other ops: two sets (select = 0 / 1) of 12 f32x2 pairs each: (re, re),
// (im, im), (-im, -im) for U00, U01, U10, U11 of a general op, or for d0 and
// d1 of a diagonal op. Where the two packed lanes (tile qubit 0 = 0 / 1) need
// different values -- a select or a diagonal target on register bit 3 -- the
// lanes are resolved here: lane 0 gets the qubit-0 = 0 value, lane 1 the
// qubit-0 = 1 value, and only set 0 is used.
// complex128: two sets of 8 doubles (re, im of U00, U01, U10, U11).
#pragma once

#include <stdint.h>

#include <complex>
#include <cstring>

#include "planner.h"

namespace qv {

inline uint64_t pack_f32x2(float lo, float hi)
{
    uint32_t a, b;
    std::memcpy(&a, &lo, 4);
    std::memcpy(&b, &hi, 4);
    return uint64_t(a) | (uint64_t(b) << 32);
}

// (re, im, -im) of z0 in lane 0 and z1 in lane 1
inline void lane_triple(uint64_t *dst, std::complex<double> z0, std::complex<double> z1)
{
    dst[0] = pack_f32x2(float(z0.real()), float(z1.real()));
    dst[1] = pack_f32x2(float(z0.imag()), float(z1.imag()));
    dst[2] = pack_f32x2(float(-z0.imag()), float(-z1.imag()));
}

// Coefficient slots (u64) an op takes in the compiled complex64 kernel: two
// sets of 12 for a 2x2 op, 48 for a GEN2 (16 entries, one set).
inline int coef_slots_c64(const plan::Op &op) { return op.type == plan::OP_GEN2 ? 48 : 24; }

// Writes coef_slots_c64(op) values.
inline void op_coeffs_c64(const plan::Op &op, uint64_t *out)
{
    if (op.type == plan::OP_GEN2) {
        for (int e = 0; e < 16; ++e) lane_triple(out + 3 * e, op.M4[e], op.M4[e]);
        return;
    }
    std::memset(out, 0, 24 * sizeof(uint64_t));
    if (op.type == plan::OP_DIAG) {
        if (op.sreg == 3) {  // select on the lane bit: lane 0 = select 0, lane 1 = select 1
            lane_triple(out, op.M[0][0], op.M[1][0]);
            lane_triple(out + 3, op.M[0][3], op.M[1][3]);
            return;
        }
        for (int s = 0; s < 2; ++s) {
            uint64_t *c = out + 12 * s;
            if (op.treg == 3) {  // target on the lane bit: lane 0 takes d0, lane 1 d1
                lane_triple(c, op.M[s][0], op.M[s][3]);
            } else {
                lane_triple(c, op.M[s][0], op.M[s][0]);
                lane_triple(c + 3, op.M[s][3], op.M[s][3]);
            }
        }
        return;
    }
    for (int e = 0; e < 4; ++e) {
        if (op.sreg == 3) {
            lane_triple(out + 3 * e, op.M[0][e], op.M[1][e]);
        } else {
            lane_triple(out + 3 * e, op.M[0][e], op.M[0][e]);
            lane_triple(out + 12 + 3 * e, op.M[1][e], op.M[1][e]);
        }
    }
}

inline void op_coeffs_c128(const plan::Op &op, double out[16])
{
    for (int s = 0; s < 2; ++s)
        for (int e = 0; e < 4; ++e) {
            out[8 * s + 2 * e] = op.M[s][e].real();
            out[8 * s + 2 * e + 1] = op.M[s][e].imag();
        }
}

}  // namespace qv
