// lbs_d3q19.cuh — the D3Q19 lattice of App. A (arXiv 2311.15242): velocity
// set, weights, the raw-moment transformation matrix of Eq. 39 with its
// inverse in closed form, and the moment equilibria of Eq. 40.
#pragma once

namespace lbs {

constexpr int Q19 = 19;

// Velocity order carried by the momentum rows of Eq. 39 (rows j_x, j_y,
// j_z): rest; +x, -x; +y, -y; +z, -z; then the xy, xz and yz diagonals, each
// as (+,+), (-,-), (+,-), (-,+).  Weights 1/3, 1/18, 1/36.
__host__ __device__ constexpr int ex19(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13)    ? 1
           : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1
                                                                  : 0;
}
__host__ __device__ constexpr int ey19(int i) {
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17)  ? 1
           : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1
                                                                 : 0;
}
__host__ __device__ constexpr int ez19(int i) {
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18)  ? 1
           : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1
                                                                   : 0;
}
// the directions come in opposite pairs (1,2), (3,4), ..., (17,18)
__host__ __device__ constexpr int opp19(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
// the direction of i mirrored on the axes of bit mask m (bits x, y, z)
__host__ __device__ constexpr int mir19c(int i, int m) {
    int r = i;
    for (int k = 0; k < 19; k++)
        if (ex19(k) == ((m & 1) ? -ex19(i) : ex19(i)) &&
            ey19(k) == ((m & 2) ? -ey19(i) : ey19(i)) && ez19(k) == ((m & 4) ? -ez19(i) : ez19(i)))
            r = k;
    return r;
}
// (with i a compile-time constant each candidate folds to a constant and the
// choice is a chain of selects: no branch, so the loads that use the result
// stay in flight together)
__host__ __device__ __forceinline__ int mir19(int i, int m) {
    const int a = (m & 1) ? mir19c(i, 1) : i, b = (m & 1) ? mir19c(i, 3) : mir19c(i, 2);
    const int c = (m & 1) ? mir19c(i, 5) : mir19c(i, 4), d = (m & 1) ? mir19c(i, 7) : mir19c(i, 6);
    return (m & 4) ? ((m & 2) ? d : c) : ((m & 2) ? b : a);
}
template <typename R>
__host__ __device__ constexpr R w19(int i) {
    return i == 0 ? R(1.0 / 3.0) : (i <= 6 ? R(1.0 / 18.0) : R(1.0 / 36.0));
}

// Rows of M (Eq. 39) as polynomials of e_i = (x, y, z):
//   0: 1            1-3: x, y, z          4: x^2 + y^2 + z^2
//   5: 2x^2-y^2-z^2  6: y^2 - z^2          7-9: xy, xz, yz
//   10-15: x^2 y, x y^2, x^2 z, x z^2, y^2 z, y z^2
//   16-18: x^2 y^2, x^2 z^2, y^2 z^2
__host__ __device__ constexpr int m19(int j, int i) {
    const int x = ex19(i), y = ey19(i), z = ez19(i);
    switch (j) {
    case 0: return 1;
    case 1: return x;
    case 2: return y;
    case 3: return z;
    case 4: return x * x + y * y + z * z;
    case 5: return 2 * x * x - y * y - z * z;
    case 6: return y * y - z * z;
    case 7: return x * y;
    case 8: return x * z;
    case 9: return y * z;
    case 10: return x * x * y;
    case 11: return x * y * y;
    case 12: return x * x * z;
    case 13: return x * z * z;
    case 14: return y * y * z;
    case 15: return y * z * z;
    case 16: return x * x * y * y;
    case 17: return x * x * z * z;
    default: return y * y * z * z;
    }
}

// f = M^{-1} m.  M is not orthogonal (row 4 and rows 16-18 overlap rows 0,
// 5, 6), but its inverse is sparse: each diagonal direction of a coordinate
// plane is fixed by that plane's xy-type, x^2 y-type and x^2 y^2-type moments;
// an axis direction by its momentum, the second-order rows and its two
// third- and fourth-order neighbours; the rest population by the remainder.
// (Obtained by solving M f = m for the symmetric and antisymmetric parts of
// each opposite pair.)
template <typename R>
__host__ __device__ __forceinline__ void minv19(const R *m, R *f) {
    const R h = R(0.5), q = R(0.25), s6 = R(1) / R(6), s12 = R(1) / R(12);
    f[0] = m[0] - m[4] + m[16] + m[17] + m[18];
    const R ax = s6 * m[4] + s6 * m[5] - h * (m[16] + m[17]);
    const R bx = h * (m[1] - m[11] - m[13]);
    f[1] = ax + bx;
    f[2] = ax - bx;
    const R ay = s6 * m[4] - s12 * m[5] + q * m[6] - h * (m[16] + m[18]);
    const R by = h * (m[2] - m[10] - m[15]);
    f[3] = ay + by;
    f[4] = ay - by;
    const R az = s6 * m[4] - s12 * m[5] - q * m[6] - h * (m[17] + m[18]);
    const R bz = h * (m[3] - m[12] - m[14]);
    f[5] = az + bz;
    f[6] = az - bz;
    // xy diagonal (sx, sy): (m16 + sx sy m7 + sy m10 + sx m11) / 4
    f[7] = q * (m[16] + m[7] + m[10] + m[11]);
    f[8] = q * (m[16] + m[7] - m[10] - m[11]);
    f[9] = q * (m[16] - m[7] - m[10] + m[11]);
    f[10] = q * (m[16] - m[7] + m[10] - m[11]);
    // xz diagonal (sx, sz): (m17 + sx sz m8 + sz m12 + sx m13) / 4
    f[11] = q * (m[17] + m[8] + m[12] + m[13]);
    f[12] = q * (m[17] + m[8] - m[12] - m[13]);
    f[13] = q * (m[17] - m[8] - m[12] + m[13]);
    f[14] = q * (m[17] - m[8] + m[12] - m[13]);
    // yz diagonal (sy, sz): (m18 + sy sz m9 + sz m14 + sy m15) / 4
    f[15] = q * (m[18] + m[9] + m[14] + m[15]);
    f[16] = q * (m[18] + m[9] - m[14] - m[15]);
    f[17] = q * (m[18] - m[9] - m[14] + m[15]);
    f[18] = q * (m[18] - m[9] + m[14] - m[15]);
}

// moment equilibrium of one colour (Eq. 40): p = rho (c_s)^2 with
// (c_s)^2 = (1 - alpha)/2 in 3D; rows 17-19 of Eq. 40 (here 16-18) as printed
template <typename R>
__host__ __device__ __forceinline__ void meq19(R rho, R ux, R uy, R uz, R al, R *m) {
    const R u2 = ux * ux + uy * uy + uz * uz;
    const R p = rho * (R(0.5) * (R(1) - al));
    m[0] = rho;
    m[1] = rho * ux;
    m[2] = rho * uy;
    m[3] = rho * uz;
    m[4] = R(3) * p + rho * u2;
    m[5] = rho * (R(2) * ux * ux - uy * uy - uz * uz);
    m[6] = rho * (uy * uy - uz * uz);
    m[7] = rho * ux * uy;
    m[8] = rho * ux * uz;
    m[9] = rho * uy * uz;
    m[10] = p * uy;
    m[11] = p * ux;
    m[12] = p * uz;
    m[13] = p * ux;
    m[14] = p * uz;
    m[15] = p * uy;
    const R b = R(1) - al - u2;
    m[16] = rho * (b + R(2) * (ux * ux + uy * uy)) / R(6);
    m[17] = rho * (b + R(2) * (ux * ux + uz * uz)) / R(6);
    m[18] = rho * (b + R(2) * (uy * uy + uz * uz)) / R(6);
}

}  // namespace lbs
