// lbs_dev.cuh — device-side definitions shared by the kernels of the coupled
// LB-FD step (arXiv 2311.15242): lattice tables, the instance descriptor,
// boundary mapping and the equation of state.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace lbs {

// ---------------------------------------------------------------------------
// D2Q9 lattice.  Velocity order: the one carried by the momentum rows of the
// transformation matrix of Eq. 36 (rows j_x, j_y), so that M below is the
// printed matrix.  Weights 4/9, 1/9, 1/36.
// ---------------------------------------------------------------------------
constexpr int Q9 = 9;

__host__ __device__ constexpr int ex9(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int ey9(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr int opp9(int i) {
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5);
}
// the direction of i mirrored on the axes of bit mask m (bit 0 x, bit 1 y):
// a population crossing mirror planes comes back specularly reflected
__host__ __device__ constexpr int mir9c(int i, int m) {
    int r = i;
    for (int k = 0; k < 9; k++)
        if (ex9(k) == ((m & 1) ? -ex9(i) : ex9(i)) && ey9(k) == ((m & 2) ? -ey9(i) : ey9(i)))
            r = k;
    return r;
}
// (with i a compile-time constant every case folds to a constant)
__host__ __device__ __forceinline__ int mir9(int i, int m) {
    return m == 0 ? i : m == 1 ? mir9c(i, 1) : m == 2 ? mir9c(i, 2) : mir9c(i, 3);
}
template <typename R>
__host__ __device__ constexpr R w9(int i) {
    return i == 0 ? R(4.0 / 9.0) : (i <= 4 ? R(1.0 / 9.0) : R(1.0 / 36.0));
}
// Rows of M (Eq. 36) as the moment polynomials of e_i:
// rho, e, epsilon, j_x, q_x, j_y, q_y, p_xx, p_xy.
__host__ __device__ constexpr int m9(int j, int i) {
    // (integer arithmetic; every entry of Eq. 36 is an integer)
    return j == 0   ? 1
           : j == 1 ? -4 + 3 * (ex9(i) * ex9(i) + ey9(i) * ey9(i))
           : j == 2 ? (8 - 21 * (ex9(i) * ex9(i) + ey9(i) * ey9(i)) +
                       9 * (ex9(i) * ex9(i) + ey9(i) * ey9(i)) *
                           (ex9(i) * ex9(i) + ey9(i) * ey9(i))) / 2
           : j == 3 ? ex9(i)
           : j == 4 ? (-5 + 3 * (ex9(i) * ex9(i) + ey9(i) * ey9(i))) * ex9(i)
           : j == 5 ? ey9(i)
           : j == 6 ? (-5 + 3 * (ex9(i) * ex9(i) + ey9(i) * ey9(i))) * ey9(i)
           : j == 7 ? ex9(i) * ex9(i) - ey9(i) * ey9(i)
                    : ex9(i) * ey9(i);
}
// squared norms of the (orthogonal) rows: M^{-1} = M^T diag(1/norm)
__host__ __device__ constexpr int mnorm9(int j) {
    return j == 0 ? 9 : (j <= 2 ? 36 : (j == 3 || j == 5 ? 6 : (j == 4 || j == 6 ? 12 : 4)));
}

// ---------------------------------------------------------------------------
// Per-step control block in device memory (dynamic state read by kernels of
// a captured graph: step counter, SOR progress, conserved total, status).
// ---------------------------------------------------------------------------
constexpr int KMAX_SWEEPS = 64;
// sweeps run after the first one that meets the tolerance: the iteration
// approaches the solution from one side, and stopping at once would leave a
// remainder of the same sign every time step
constexpr int SOR_EXTRA = 2;
enum : int { ST_NOCONV = 1, ST_DIVERGED = 2, ST_TIMEOUT = 4 };

struct Ctl {
    long long step;         // time steps taken
    double M0;              // conserved total surfactant
    double pre;             // total before the last rescale
    double scale;           // last rescale factor
    int status;             // ST_* bits, sticky until read by the host
    int sor_iters;          // sweeps used by the last solve
    unsigned int ticket;    // arrival counter of the last-block reductions
    int sor_exec;           // sweeps (rounds) executed in the current solve
    int sor_iters_parity;   // rounds of the last solve were odd: result in psi2, C2
    unsigned int sor_ticket; // arrival counter of the SOR round blocks
    double dscale;          // scale - 1 of the last rescale
    float dscale_f;         // the same in single precision
    int sor_active;         // batched sweep: 1 while this instance's solve iterates
    int dead;               // non-finite total seen: a batch skips this instance
    unsigned int bar_count; // grid barrier of the one-launch SOR: arrivals
    unsigned int bar_gen;   // (unused)
    // per sweep: max |d psi|, max |d C|, max |psi|, max |C| (bits of
    // non-negative doubles, compared as unsigned integers)
    unsigned long long sweep[KMAX_SWEEPS][4];
    double diag[32];        // finalised diagnostics sums
};

// ---------------------------------------------------------------------------
// Instance descriptor passed by value to every kernel.
// ---------------------------------------------------------------------------
template <typename R>
struct Inst {
    int nx, ny, nz, pitch;   // pitch: elements per row (>= nx); cell (x, y, z) at
                             // (z ny + y) pitch + x
    long long plane;         // elements per scalar plane (pitch * ny * nz)
    int wall[3];              // per axis: 0 periodic, 1 bounce-back walls, 2 mirror planes
    int bbmask;               // bit a set where axis a has bounce-back walls
    int mvmask;               // bit a set where those walls move
    R uw_lo[3][3], uw_hi[3][3];
    R rhoR0, rhoB0, alphaR, alphaB, cs2R, cs2B, muR0, muB0;
    R inv_rhoR0, inv_rhoB0;  // 1 / rho^k0
    R inv_2muR, inv_2muB;    // 1 / (2 mu^k0)
    R beta, eps_n, eps_w;
    R sigma0, sigma_min, E0, psi_inf, cmc;
    int eos, source, transport;
    R Ds, Db, ra, rd, g[3], omega, sor_tol;
    int sor_max_iter;
    R pscale, pinv;          // storage scale of FP16 populations (a power of 2) and 1/scale
    // shift of the stored total populations: the rest equilibrium of the pure
    // majority phase of a cell.  Its moving components are common to both
    // phases (equal pure-phase pressures, Eq. 42): shift[1..Q-1]; the rest
    // component depends on the cell's flag: shift0[flag].  rho_s[flag] is the
    // sum of the shift, dsh[flag] = rho_s[flag] - rho^k0 of the majority phase.
    R shift[19];
    R shift0[2], rho_s[2], dsh[2];
    // moments of the shift minus those of the pure majority phase at rest
    // (rounding only, unless alpha breaks Eq. 42): D2Q9 rows e and epsilon of
    // Eq. 36; D3Q19 row 4 (|e|^2) and rows 16-18 (x^2 y^2 type, all equal)
    // of Eq. 39
    R mcor1[2], mcor2[2];
    int sor_pingpong;         // SOR result alternates between psi/C and psi2/C2
    int sor_phase;            // 1: round 0 of a solve reads psi2/C2 (the fused 2D
                              // step leaves the starting guess there), 0: psi/C
    int pop_pp;               // 1: the population sets alternate by the parity of the
                              // step counter (the fused 2D step); 0: set f between steps
    // state (device pointers; every field is `plane` elements, populations Q planes)
    // populations in the storage type P of the kernels that touch them
    // (float / double, or __half / __nv_bfloat16 for the shifted
    // low-precision forms): ldp / stp below convert
    void *fT, *fM;            // total populations minus shift, minority colour
    void *gT, *gM;            // post-collision buffers
    // the rest populations (i = 0) of the four sets, in R for every storage
    // form: they absorb the rounding residuals of the moving populations, so
    // that the stored populations of a cell sum to its colour masses
    R *fT0, *fM0, *gT0, *gM0;
    uint8_t *flag, *gflag;    // minority colour of a cell: 0 red, 1 blue
    R *rhoR, *rhoB, *rhoN, *jx, *jy, *jz;
    R *gx, *gy, *gz, *a, *chi;  // grad rhoN, |grad rhoN|, 1 - rhoN
    R *ux, *uy, *uz, *Fx, *Fy, *Fz;  // z components: D3Q19 only (null in 2D)
    R *psi, *C, *S, *B, *rpsi, *rC;
    R *psi2, *C2;             // second buffers of the blocked SOR rounds
    R *psip, *Cp;             // psi, C of the previous time level (SOR initial guess)
    // the fused 2D step: moments of t+1 (rho^R, rho^B, rho^N, j), written while
    // neighbouring tiles still read those of t (null otherwise)
    R *rhoRn, *rhoBn, *rhoNn, *jxn, *jyn;
    // 2D: the coefficients of the step's CN systems, written by the first SOR
    // round and read by the later ones: faces towards +x and +y of the psi
    // and C systems and their inverse diagonals (null in 3D)
    R *sfx, *sfy, *scx, *scy, *sip, *sic;
    Ctl *ctl;
    double *part;             // per-block partial sums of reductions
};

// The moment planes rho^R, rho^B, rho^N, j of one set.  The fused 2D step
// keeps those of step s in set s & 1, like its populations (it reads one set
// and writes the other, so nothing is copied); the other forms use set 0.
template <typename R>
struct MomSet {
    R *rR, *rB, *rN, *jx, *jy;
};
template <typename R>
__host__ __device__ __forceinline__ MomSet<R> mom_set(const Inst<R> &I, bool second) {
    return second ? MomSet<R>{I.rhoRn, I.rhoBn, I.rhoNn, I.jxn, I.jyn}
                  : MomSet<R>{I.rhoR, I.rhoB, I.rhoN, I.jx, I.jy};
}
// the set that holds the moments of step s
template <typename R>
__host__ __device__ __forceinline__ MomSet<R> mom_of_step(const Inst<R> &I, long long s) {
    return mom_set(I, I.pop_pp && (s & 1));
}

// ---------------------------------------------------------------------------
// Population storage: arithmetic in R, storage in P.  The stored numbers are
// deviations from a rest state or minority-colour populations, all small,
// which is what makes 16-bit storage usable.
// ---------------------------------------------------------------------------
// FP16 populations are stored multiplied by a power of two (2^14 for pure-
// phase densities <= 1, lower for heavier phases, set on the host): the
// interface tails carry minority populations of 1e-7..1e-4, which unscaled
// FP16 keeps only as subnormals; scaled, its normal range reaches ~4e-9.
template <typename P>
struct PopCvt;
template <>
struct PopCvt<float> {
    static constexpr bool scaled = false;
    static __device__ __forceinline__ float to(float v) { return v; }
    static __device__ __forceinline__ float from(float v) { return v; }
    static __device__ __forceinline__ float from_r(float v, unsigned int) { return v; }
};
template <>
struct PopCvt<double> {
    static constexpr bool scaled = false;
    static __device__ __forceinline__ double to(double v) { return v; }
    static __device__ __forceinline__ double from(double v) { return v; }
    static __device__ __forceinline__ double from_r(double v, unsigned int) { return v; }
};
template <>
struct PopCvt<__half> {
    static constexpr bool scaled = true;
    static __device__ __forceinline__ float to(__half v) { return __half2float(v); }
    static __device__ __forceinline__ __half from(float v) { return __float2half_rn(v); }
    // one of the two neighbouring values, the far one with probability by
    // distance (r: 32 uniform bits): the top bits of r are added to the bits
    // of v that the rounding drops, and their carry decides, so the
    // probability is exactly the dropped fraction.  Integer instructions
    // only, no branch: v's significand m (leading one included) counts
    // steps of 2^(e - 150) for its exponent field e; FP16's step is
    // 2^(max(e, 113) - 137), t = 126 - min(e, 113) bits coarser (13 in
    // FP16's normal range, more in its subnormal range below 2^-14).  The
    // rounded count k is the FP16 significand (1024..2048, a carry being the
    // next binade's first value) or, below 2^-14, the whole FP16 number.
    // Exact for t <= 31 (|v| >= 2^-32); below, m is first shifted down to 31
    // bits, which lowers the probability by less than 2^-31.
    static __device__ __forceinline__ __half from_r(float v, unsigned int r) {
        const unsigned int b = __float_as_uint(v), a = b & 0x7FFFFFFFu;
        const unsigned int e = max(a >> 23, 1u);
        const unsigned int m = (a & 0x7FFFFFu) | (a >= 0x800000u ? 0x800000u : 0u);
        const unsigned int t = 126u - min(e, 113u), tt = min(t, 31u);
        const unsigned int k = ((m >> min(t - tt, 31u)) + (r >> (32u - tt))) >> tt;
        const unsigned int h = ((max(e, 113u) - 113u) << 10) + k;
        return __ushort_as_half((unsigned short)(h | ((b >> 16) & 0x8000u)));
    }
};
template <>
struct PopCvt<__nv_bfloat16> {
    static constexpr bool scaled = false;
    static __device__ __forceinline__ float to(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ __nv_bfloat16 from(float v) { return __float2bfloat16_rn(v); }
    // as FP16's: BF16 is FP32 without the low 16 bits, at every magnitude
    static __device__ __forceinline__ __nv_bfloat16 from_r(float v, unsigned int r) {
        return __ushort_as_bfloat16((unsigned short)((__float_as_uint(v) + (r >> 16)) >> 16));
    }
};

template <typename R, typename P>
__device__ __forceinline__ R ldp(const Inst<R> &I, const void *base, long long k) {
    R v = R(PopCvt<P>::to(((const P *)base)[k]));
    return PopCvt<P>::scaled ? v * I.pinv : v;
}
template <typename R, typename P>
__device__ __forceinline__ void stp(const Inst<R> &I, void *base, long long k, R v) {
    ((P *)base)[k] = PopCvt<P>::from(PopCvt<P>::scaled ? v * I.pscale : v);
}

// population i of cell c of a set (moving array mov, rest plane rest)
template <typename R, typename P>
__device__ __forceinline__ R ldq(const Inst<R> &I, const void *mov, const R *rest, int i,
                                 long long c) {
    return i == 0 ? rest[c] : ldp<R, P>(I, mov, (long long)i * I.plane + c);
}
// store moving population i (i >= 1); returns the value actually stored
template <typename R, typename P>
__device__ __forceinline__ R stq(const Inst<R> &I, void *mov, int i, long long c, R v) {
    const P s = PopCvt<P>::from(PopCvt<P>::scaled ? v * I.pscale : v);
    ((P *)mov)[(long long)i * I.plane + c] = s;
    const R back = R(PopCvt<P>::to(s));
    return PopCvt<P>::scaled ? back * I.pinv : back;
}
// the same, rounded to a 16-bit storage without bias (r: the population's
// draw, pop_r); FP32 and FP64 storage store v itself
template <typename R, typename P>
__device__ __forceinline__ R stq_r(const Inst<R> &I, void *mov, int i, long long c, R v,
                                   unsigned int r) {
    const P s = PopCvt<P>::from_r(PopCvt<P>::scaled ? v * I.pscale : v, r);
    ((P *)mov)[(long long)i * I.plane + c] = s;
    const R back = R(PopCvt<P>::to(s));
    return PopCvt<P>::scaled ? back * I.pinv : back;
}

// error-free transformations (Knuth's TwoSum): a + b = s + e exactly
template <typename R>
__device__ __forceinline__ R two_sum(R a, R b, R &e) {
    const R s = a + b;
    const R bp = s - a;
    e = (a - (s - bp)) + (b - bp);
    return s;
}

// ---------------------------------------------------------------------------
// Boundary mapping.  Periodic axes wrap; on a walled axis the coordinate is
// mirrored about the half-way wall (-1 -> 0, -2 -> 1, n -> n-1, ...).
// refl: bit a set when axis a was reflected; side: -1 low wall, +1 high wall.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int map_axis(int c, int n, int wall, int bit, int &refl,
                                        int &side) {
    side = 0;
    if (c >= 0 && c < n) return c;
    if (!wall) return ((c % n) + n) % n;
    refl |= bit;
    if (c < 0) {
        side = -1;
        return -1 - c;
    }
    side = 1;
    return 2 * n - 1 - c;
}

// the mapped coordinates of offsets -2..2 along one axis, computed once per
// thread: v (coordinate), r (reflection bit of the axis or 0), s (wall side)
struct Ax {
    int v[5];
    unsigned char r[5];
    signed char s[5];
};
__device__ __forceinline__ Ax make_ax(int c, int n, int wall, int bit) {
    Ax a;
#pragma unroll
    for (int k = 0; k < 5; k++) {
        int refl = 0, side;
        a.v[k] = map_axis(c + k - 2, n, wall, bit, refl, side);
        a.r[k] = (unsigned char)refl;
        a.s[k] = (signed char)side;
    }
    return a;
}
// neighbour (dx, dy) of a 2D cell from its axes (|d| <= 2)
template <typename R>
__device__ __forceinline__ long long nbx2(const Inst<R> &I, const Ax &X, const Ax &Y, int dx,
                                          int dy, int &refl, int &sx, int &sy) {
    refl = X.r[dx + 2] | Y.r[dy + 2];
    sx = X.s[dx + 2];
    sy = Y.s[dy + 2];
    return (long long)Y.v[dy + 2] * I.pitch + X.v[dx + 2];
}
// neighbour (dx, dy, dz) of a 3D cell from its axes
template <typename R>
__device__ __forceinline__ long long nbx3(const Inst<R> &I, const Ax &X, const Ax &Y, const Ax &Z,
                                          int dx, int dy, int dz, int &refl, int &sx, int &sy,
                                          int &sz) {
    refl = X.r[dx + 2] | Y.r[dy + 2] | Z.r[dz + 2];
    sx = X.s[dx + 2];
    sy = Y.s[dy + 2];
    sz = Z.s[dz + 2];
    return ((long long)Z.v[dz + 2] * I.ny + Y.v[dy + 2]) * I.pitch + X.v[dx + 2];
}

// programmatic dependent launch.  A kernel launched as the programmatic
// dependent of the kernel before it in the stream waits in pdl_wait until
// that kernel has finished and its writes are visible; for an ordinary launch
// pdl_wait returns at once.  pdl_trigger lets the dependent grid launch (its
// blocks then wait in pdl_wait) once every block of this grid has run it, so
// its launch overlaps this grid's tail.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;"); }

// two consecutive elements (one aligned vector load or store)
template <typename R>
struct Vec2;
template <>
struct Vec2<float> {
    using T = float2;
};
template <>
struct Vec2<double> {
    using T = double2;
};

// ---------------------------------------------------------------------------
// The rescale of the total surfactant (Sec. 2.2) applied to one value:
// x (1 + d) with d = s - 1 = O(1e-7).  In double precision one fused
// rounding.  In single precision x d is one or two ulps of x, and rounding
// x + x d to nearest errs the same way in every cell whose value and
// exponent agree (the whole bulk liquid), a bias of the rescaled total of up
// to half an ulp each step; instead the result is one of the two floats
// around x + x d (formed exactly as s + e by TwoSum), the far one with
// probability |e| / ulp, so the rounding error is zero on average.  The draw
// is MurmurHash3's 32-bit finaliser (Appleby) of the cell, the field and the
// step: reproducible, a restarted run draws the same.  FP32 arithmetic only
// (the FP64 pipe of GB300 is narrow).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned int fmix32(unsigned int h) {
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}
// the draw of cell c, field k (0 psi, 1 C), step n
__device__ __forceinline__ unsigned int rescale_key(long long c, int k, long long n) {
    return fmix32((unsigned int)c ^ fmix32((unsigned int)(2 * n + k)));
}
// the exact s + e (s = fl(s + e), |e| <= ulp/2) rounded without bias: s, or
// its neighbour on the side of e with probability |e| / (distance to it)
__device__ __forceinline__ float pick_unbiased(float s, float e, unsigned int key) {
    if (e == 0.0f) return s;
    const float nb = nextafterf(s, e > 0.0f ? INFINITY : -INFINITY);
    const float frac = __fdividef(e, nb - s);  // in (0, 1/2]
    const float u = float(key >> 8) * 0x1.0p-24f;
    return u < frac ? nb : s;
}
__device__ __forceinline__ double rescale_one(double x, double d, float, unsigned int) {
    return fma(x, d, x);
}
__device__ __forceinline__ float rescale_one(float x, double, float d, unsigned int key) {
    float e;
    const float s = two_sum(x, x * d, e);
    return pick_unbiased(s, e, key);
}

// ---------------------------------------------------------------------------
// A cell's rest population closes its mass: (a_s + a_c) - (b_s + b_c) + lo,
// the difference of two compensated sums (the mass the cell holds, the mass
// its stored moving populations carry) plus a small term.  The hi parts are
// subtracted exactly (TwoSum), so the value is exact before the one rounding
// to the storage; in single precision that rounding is unbiased (as the
// rescale's above).  Rounding to nearest erred the same way step after step:
// on a steady interface a cell receives the same sub-ulp residual of its
// 16-bit moving populations every step, and rounding dropped it every time,
// moving about 1e-9 of one colour's mass into the other's a cell and step.
// The draws: one 32-bit hash of the cell and a salt of the kernel and step
// (rest_salt, the same for every cell of a launch) gives the cell's two
// closures (total, minority) a 16-bit uniform each (rest_u).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned int rest_salt(int tag, long long n) {
    return fmix32((unsigned int)(4 * n + tag) ^ 0x9E3779B9u);
}
__device__ __forceinline__ unsigned int rest_key(long long c, unsigned int salt) {
    return fmix32((unsigned int)c ^ salt);
}
// uniform in [0, 1) of half h (0: total, 1: minority) of a cell's key
__device__ __forceinline__ float rest_u(unsigned int key, int h) {
    return float(h ? key >> 16 : key & 0xFFFFu) * 0x1.0p-16f;
}
// The moving populations' 16-bit storage is rounded without bias too, since
// at a steady interface rounding to nearest errs the same way every step.
// Their draws: a second hash of the cell's key (pop_seed, mixed apart from
// the closures' draws), times an odd constant for population j (2 i for the
// total, 2 i + 1 for the minority): a bijection of 32-bit words, so each
// draw is uniform, at one multiply a population.
__device__ __forceinline__ unsigned int pop_seed(unsigned int key) {
    return fmix32(key ^ 0x85EBCA6Bu);
}
__device__ __forceinline__ unsigned int pop_r(unsigned int seed, int j) {
    return seed * (0x9E3779B9u * (2u * (unsigned int)j + 1u));
}
__device__ __forceinline__ double rest_close(double as, double ac, double bs, double bc,
                                             double lo, float) {
    double e;
    const double d = two_sum(as, -bs, e);
    return d + ((e + (ac - bc)) + lo);
}
__device__ __forceinline__ float rest_close(float as, float ac, float bs, float bc, float lo,
                                            float u) {
    float e1, e2;
    const float d = two_sum(as, -bs, e1);
    const float s = two_sum(d, (e1 + (ac - bc)) + lo, e2);
    if (e2 == 0.0f) return s;
    const float nb = nextafterf(s, e2 > 0.0f ? INFINITY : -INFINITY);
    return u < __fdividef(e2, nb - s) ? nb : s;
}

// the product a b exactly as hi + lo (lo by one FMA), added to a compensated
// sum (hi, lo): the total surfactant of the rescale to about 1e-14 in FP32
// arithmetic
__device__ __forceinline__ void comp_add_prod(float &hi, float &lo, float a, float b) {
    const float p = a * b;
    const float pe = fmaf(a, b, -p);
    float e;
    hi = two_sum(hi, p, e);
    lo += e + pe;
}
__device__ __forceinline__ void comp_add_prod(double &hi, double &lo, double a, double b) {
    const double p = a * b;
    const double pe = fma(a, b, -p);
    double e;
    hi = two_sum(hi, p, e);
    lo += e + pe;
}

// division and inverse square root: IEEE in double precision; in single
// precision the hardware approximations (about 2 ulp), whose errors are of
// the order of the FP32 rounding of the stored fields
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double frsq(double a) { return 1.0 / sqrt(a); }
__device__ __forceinline__ float frsq(float a) { return rsqrtf(a); }

template <typename R>
__device__ __forceinline__ long long nb2(const Inst<R> &I, int x, int y, int dx, int dy,
                                         int &refl, int &sx, int &sy) {
    refl = 0;
    int X = map_axis(x + dx, I.nx, I.wall[0], 1, refl, sx);
    int Y = map_axis(y + dy, I.ny, I.wall[1], 2, refl, sy);
    return (long long)Y * I.pitch + X;
}

// velocity at a ghost node: u -> 2 u_wall - u for each wall crossed
template <typename R>
__device__ __forceinline__ void ghost_u2(const Inst<R> &I, int refl, int sx, int sy,
                                         R &u0, R &u1) {
    // a mirror plane reflects the normal component only (free slip)
    if (refl & ~I.bbmask & 1) {
        u0 = -u0;
        refl &= ~1;
    }
    if (refl & ~I.bbmask & 2) {
        u1 = -u1;
        refl &= ~2;
    }
    if (refl & 1) {
        const R *w = sx < 0 ? I.uw_lo[0] : I.uw_hi[0];
        u0 = R(2) * w[0] - u0;
        u1 = R(2) * w[1] - u1;
    }
    if (refl & 2) {
        const R *w = sy < 0 ? I.uw_lo[1] : I.uw_hi[1];
        u0 = R(2) * w[0] - u0;
        u1 = R(2) * w[1] - u1;
    }
}

// 3D neighbour (same wall mapping per axis; bit 4 for z)
template <typename R>
__device__ __forceinline__ long long nb3(const Inst<R> &I, int x, int y, int z, int dx, int dy,
                                         int dz, int &refl, int &sx, int &sy, int &sz) {
    refl = 0;
    int X = map_axis(x + dx, I.nx, I.wall[0], 1, refl, sx);
    int Y = map_axis(y + dy, I.ny, I.wall[1], 2, refl, sy);
    int Z = map_axis(z + dz, I.nz, I.wall[2], 4, refl, sz);
    return ((long long)Z * I.ny + Y) * I.pitch + X;
}

template <typename R>
__device__ __forceinline__ long long cell3(const Inst<R> &I, int x, int y, int z) {
    return ((long long)z * I.ny + y) * I.pitch + x;
}

// 3D ghost velocity: u -> 2 u_wall - u for each wall crossed
template <typename R>
__device__ __forceinline__ void ghost_u3(const Inst<R> &I, int refl, int sx, int sy, int sz,
                                         R &u0, R &u1, R &u2) {
    const int side[3] = {sx, sy, sz};
    // a mirror plane reflects the normal component only (free slip)
    if (refl & ~I.bbmask & 1) u0 = -u0;
    if (refl & ~I.bbmask & 2) u1 = -u1;
    if (refl & ~I.bbmask & 4) u2 = -u2;
    refl &= I.bbmask;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        if (!(refl & (1 << a))) continue;
        const R *w = side[a] < 0 ? I.uw_lo[a] : I.uw_hi[a];
        u0 = R(2) * w[0] - u0;
        u1 = R(2) * w[1] - u1;
        u2 = R(2) * w[2] - u2;
    }
}

// ---------------------------------------------------------------------------
// Equation of state (Eq. 8) and the Marangoni coefficient -d sigma/d psi of
// Eq. 9.  Above the CMC sigma = sigma_min and the coefficient is 0.  The
// logarithm is taken in double precision near saturation (psi/psi_inf > 1/2).
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ bool eos(const Inst<R> &I, R psi, R &sigma, R &mcoef) {
    if (I.E0 == R(0)) {  // Eq. 8 with E0 = 0: constant tension
        sigma = I.sigma0;
        mcoef = R(0);
        return true;
    }
    if (I.eos == 1) {
        sigma = I.sigma0 * (R(1) - I.E0 * psi / I.psi_inf);
        mcoef = I.sigma0 * I.E0 / I.psi_inf;
        return true;
    }
    if (psi < I.cmc) {
        R x = -psi / I.psi_inf;
        R lg;
        if (x < R(-0.5))
            lg = R(log1p(double(x)));
        else
            lg = log1p(x);
        sigma = I.sigma0 * (R(1) + I.E0 * lg);
        mcoef = I.sigma0 * I.E0 / (I.psi_inf - psi);
        return true;
    }
    sigma = I.sigma_min;
    mcoef = R(0);
    return false;
}

}  // namespace lbs
