/*
 * GBEES oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow FP64 CPU implementation of the per-step
 * propagation of a probability density on a sparse Cartesian grid, as
 * described in "GBEES-GPU: An efficient parallel GPU algorithm for
 * high-dimensional nonlinear uncertainty propagation" (Hanson, Rubio,
 * Garcia-Gutierrez, Bewley; arXiv 2508.13986).
 *
 * Only the test-suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this library. It shares no code, header, table or helper with the
 * CUDA library in paper_2508_13986_gb300/, and neither includes the other.
 *
 * Structure (one function per step of the method, in the paper's order):
 *   dynamics f(x)                      Sec. 5.1.1 (Lorenz '63), Sec. 5.1.2 (Lorenz '96)
 *   face velocity f_j(x_{i-e_j/2})     Eq. 7 (the velocity that enters DCU)
 *   initial Gaussian                   Sec. 5.1 (the initial PDFs)
 *   directional grow / prune           Sec. 3.3, Figs. 2-3, Algorithm 3
 *   CFL time step                      Eq. 8 (with |f| and the CFL number of Sec. 5.2.2)
 *   DCU flux                           Eq. 7
 *   CTU transverse corrections         Algorithm 1
 *   high-resolution correction         Sec. 2.1 (deferred by the paper to Bewley & Sharma)
 *   conservative update                Eq. 3 discretised over V_i (Eqs. 5-6)
 *   normalisation                      Sec. 4.3 / 4.5
 *   Bayesian measurement update        Eq. 4
 *
 * Readings of points the paper leaves open (the CUDA library follows the same):
 *   - Lorenz '63 is available both in the classic form (sigma, rho, beta) and in
 *     the shifted form the paper prints in Sec. 5.1.1 (sigma, b, r).
 *   - Eq. 8 is read with |f| and multiplied by the CFL number:
 *       dt = CFL / max_i sum_j |f_j(x_{i-e_j/2})| / h_j,
 *     over every active cell after grow, clipped so that t lands on the target
 *     time exactly; a grid whose rates are all zero takes the whole interval.
 *   - "significant" means p > thr_rel * max p (strict).
 *   - The downwind set D(i) of a cell holds the face neighbours across every
 *     face whose velocity points out of i, plus the edge neighbours reached by
 *     two such outward steps in two different dimensions (the CTU stencil is
 *     pairwise). Grow inserts D(S) with p = 0 for S = significant cells.
 *   - Prune keeps S u D(S) (the mirror image of grow: a cell below threshold
 *     survives only if an upwind significant neighbour would grow into it).
 *     It runs every `prune_interval` steps and after every measurement update,
 *     before the normalisation, so that every returned density integrates to one.
 *   - The grid is conceptually infinite with P = 0 off the active set. DCU
 *     fluxes, the waves of Algorithm 1 and the high-resolution corrections are
 *     evaluated on every face that touches an active cell; only active cells are
 *     updated, so flux into a missing cell is lost and normalisation restores
 *     the total.
 *   - High-resolution correction (wave limiting in the form of LeVeque's
 *     "Finite Volume Methods for Hyperbolic Problems", Ch. 6 and 20):
 *       F_{X,j} += 1/2 |u| (1 - dt |u| / h_j) phi(theta) W,
 *       W = P_X - P_{X-e_j},  theta = W_upwind / W,
 *     the upwind wave taken at the face below (u > 0) or above (u < 0); the
 *     MC limiter phi(theta) = max(0, min((1+theta)/2, 2, 2 theta)) by default;
 *     NONE (phi = 0) and LW (phi = 1) are test modes; W = 0 adds nothing. The
 *     correction is not propagated transversely.
 *   - The density (not the cell mass) is stored and normalised so that
 *     (prod_j h_j) sum_i p_i = 1; the sum is exact (a fixed-point
 *     superaccumulator) so that it does not depend on the order of the cells.
 *   - The grid origin x0 is part of the configuration; cell i has centre
 *     x0 + i * h and its lower face in dimension j sits at x0_j + (i_j - 1/2) h_j.
 *
 * Threads: loops over cells and faces may run in parallel (OpenMP, when the
 * library is built with it). Each parallel iteration writes only its own slot,
 * maxima are order-free, the exact sums are merged digit by digit, and every
 * floating-point sum whose rounding depends on its order is accumulated in
 * the order of the single-threaded program (the transverse corrections of one
 * flux array by one thread, in the order of the faces that emit them; cells
 * and faces are inserted into the maps in the same order). The results are
 * therefore the same for any number of threads.
 *
 * Compile with -ffp-contract=off so that no multiply-add is fused.
 */
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

enum { DYN_CONSTANT = 0, DYN_LINEAR = 1, DYN_LORENZ63 = 2, DYN_LORENZ63_SHIFTED = 3, DYN_LORENZ96 = 4 };
enum { LIM_MC = 0, LIM_NONE = 1, LIM_LW = 2 };
enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_EDEGENERATE = -4 };

}  // namespace

extern "C" {
/* The oracle's own configuration record (declared here only; the CUDA
 * library declares its own). */
typedef struct {
    int32_t n;              /* dimension, 1..6 */
    int32_t dynamics;       /* DYN_* above */
    double params[64];      /* model parameters */
    double h[6];            /* cell widths */
    double x0[6];           /* centre of cell 0 */
    double thr_rel;         /* significance threshold relative to max p */
    double cfl;             /* CFL number */
    int32_t prune_interval; /* prune every K steps */
    int32_t limiter;        /* LIM_* above */
} orc_config;

typedef struct {
    int64_t steps;        /* steps taken by the last propagate call */
    int64_t cell_updates; /* sum over those steps of the active-cell count */
    double t;             /* time reached */
    double last_dt;       /* the last step's dt */
    int64_t total_steps;  /* steps since init */
} orc_stats;
}

namespace {

using Idx = std::array<int32_t, 6>;

struct IdxHash {
    size_t operator()(const Idx& a) const {
        uint64_t x = 0x9E3779B97F4A7C15ull;
        for (int k = 0; k < 6; ++k) {
            x ^= (uint64_t)(uint32_t)a[k];
            x *= 0xBF58476D1CE4E5B9ull;
            x ^= x >> 31;
        }
        return (size_t)x;
    }
};

using Field = std::unordered_map<Idx, double, IdxHash>;

/* ---------------------------------------------------------------------------
 * Exact sum of doubles: a fixed-point integer whose unit is 2^-1074 (the
 * smallest subnormal), wide enough for every finite double, held as signed
 * 32-bit digits in 64-bit cells so that up to 2^31 additions need no carry.
 * The result is the exact sum rounded once to nearest-even.
 * ------------------------------------------------------------------------- */
struct ExactSum {
    static const int NDIG = 70; /* 70 * 32 = 2240 bits > 1074 + 1024 + 64 */
    int64_t d[NDIG];
    ExactSum() { std::memset(d, 0, sizeof d); }

    void add(double x) {
        if (x == 0.0) return;
        int e = 0;
        double m = std::frexp(std::fabs(x), &e);           /* |x| = m 2^e, m in [0.5, 1) */
        uint64_t mi = (uint64_t)std::ldexp(m, 53);         /* exact 53-bit integer */
        int pos = e - 53 + 1074;                           /* |x| = mi * 2^(pos - 1074) */
        if (pos < 0) { mi >>= -pos; pos = 0; }             /* subnormal input: exact shift */
        int k = pos / 32, r = pos % 32;
        unsigned __int128 v = (unsigned __int128)mi << r;
        int64_t sgn = x < 0 ? -1 : 1;
        for (int q = 0; q < 3 && k + q < NDIG; ++q) {
            d[k + q] += sgn * (int64_t)(uint32_t)(v >> (32 * q));
        }
    }

    /* add another exact sum (digit by digit: exact, in any order) */
    void merge(const ExactSum& o) {
        for (int q = 0; q < NDIG; ++q) d[q] += o.d[q];
    }

    double value() const {
        /* carry-normalise into base-2^32 digits with a signed top */
        int64_t c[NDIG];
        std::memcpy(c, d, sizeof c);
        for (int k = 0; k < NDIG - 1; ++k) {
            int64_t carry = c[k] >> 32; /* arithmetic shift = floor division */
            c[k] -= carry * ((int64_t)1 << 32);
            c[k + 1] += carry;
        }
        bool neg = c[NDIG - 1] < 0;
        uint32_t mag[NDIG];
        if (neg) {
            /* magnitude of a two's complement number: invert and add one */
            uint64_t carry = 1;
            for (int k = 0; k < NDIG; ++k) {
                uint64_t w = (uint64_t)(uint32_t)(~(uint32_t)c[k]) + carry;
                mag[k] = (uint32_t)w;
                carry = w >> 32;
            }
        } else {
            for (int k = 0; k < NDIG; ++k) mag[k] = (uint32_t)c[k];
        }
        int top = -1;
        for (int k = NDIG - 1; k >= 0; --k)
            if (mag[k]) { top = k; break; }
        if (top < 0) return 0.0;
        int hb = 31;
        while (!((mag[top] >> hb) & 1u)) --hb;
        int msb = 32 * top + hb; /* bit index of the leading one */
        auto bit = [&](int b) -> uint64_t { return b < 0 ? 0 : ((mag[b / 32] >> (b % 32)) & 1u); };
        double result;
        if (msb < 53) {
            uint64_t v = 0;
            for (int b = msb; b >= 0; --b) v = (v << 1) | bit(b);
            result = std::ldexp((double)v, -1074);
        } else {
            uint64_t v = 0;
            for (int b = msb; b > msb - 53; --b) v = (v << 1) | bit(b);
            uint64_t round = bit(msb - 53);
            bool sticky = false;
            for (int b = msb - 54; b >= 0 && !sticky; --b) sticky = bit(b) != 0;
            if (round && (sticky || (v & 1))) v += 1; /* v may become 2^53: still exact */
            result = std::ldexp((double)v, msb - 52 - 1074);
        }
        return neg ? -result : result;
    }
};

/* --------------------------------------------------------------------------- */

struct Oracle {
    orc_config c;
    Field P;              /* active cells and their density */
    double t = 0.0;
    int64_t step = 0;     /* steps since init */
    double last_dt = 0.0;
    double prod_h = 1.0;  /* h_1 h_2 ... h_n, multiplied in order */
    std::string err;
};

/* Drift f_j(x) of the chosen model (Sec. 5.1). */
double drift(const orc_config& c, const double* x, int j) {
    const double* a = c.params;
    switch (c.dynamics) {
        case DYN_CONSTANT:
            return a[j];
        case DYN_LINEAR: { /* f = A x + b, A row-major n x n, then b */
            double s = 0.0;
            for (int k = 0; k < c.n; ++k) s += a[j * c.n + k] * x[k];
            return s + a[c.n * c.n + j];
        }
        case DYN_LORENZ63: { /* classic form: sigma, rho, beta */
            if (j == 0) return a[0] * (x[1] - x[0]);
            if (j == 1) return x[0] * (a[1] - x[2]) - x[1];
            return x[0] * x[1] - a[2] * x[2];
        }
        case DYN_LORENZ63_SHIFTED: { /* Sec. 5.1.1: sigma, b, r */
            if (j == 0) return a[0] * (x[1] - x[0]);
            if (j == 1) return -x[1] - x[0] * x[2];
            return -a[1] * x[2] + x[0] * x[1] - a[1] * a[2];
        }
        case DYN_LORENZ96: { /* Sec. 5.1.2, cyclic indices */
            int n = c.n;
            return (x[(j + 1) % n] - x[(j + n - 2) % n]) * x[(j + n - 1) % n] - x[j] + a[0];
        }
    }
    return 0.0;
}

/* Centre of cell i in dimension k (Eq. 5). */
inline double centre(const Oracle& o, const Idx& i, int k) { return o.c.x0[k] + i[k] * o.c.h[k]; }

/* f_j at the centre of the lower face of cell X in dimension j: the velocity
 * f_{X - e_j/2, j} of Eq. 7. */
double face_velocity(const Oracle& o, const Idx& X, int j) {
    double y[6] = {0, 0, 0, 0, 0, 0};
    for (int k = 0; k < o.c.n; ++k) y[k] = centre(o, X, k);
    y[j] = o.c.x0[j] + (X[j] - 0.5) * o.c.h[j];
    return drift(o.c, y, j);
}

inline Idx shifted(Idx X, int j, int s) { X[j] += s; return X; }

inline double get(const Field& P, const Idx& X) {
    auto it = P.find(X);
    return it == P.end() ? 0.0 : it->second;
}

/* The cells of P in its iteration order (for loops that run in parallel). */
std::vector<std::pair<const Idx, double>*> cell_list(Field& P) {
    std::vector<std::pair<const Idx, double>*> v;
    v.reserve(P.size());
    for (auto& kv : P) v.push_back(&kv);
    return v;
}
std::vector<const std::pair<const Idx, double>*> cell_list(const Field& P) {
    std::vector<const std::pair<const Idx, double>*> v;
    v.reserve(P.size());
    for (auto& kv : P) v.push_back(&kv);
    return v;
}

double max_p(const Field& P) {
    const auto cells = cell_list(P);
    const int64_t N = (int64_t)cells.size();
    double m = -INFINITY;
#pragma omp parallel for reduction(max : m) schedule(static)
    for (int64_t i = 0; i < N; ++i) m = std::max(m, cells[i]->second);
    return m;
}

/* Downwind set D(i) (Sec. 3.3, Fig. 2). */
std::vector<Idx> downwind(const Oracle& o, const Idx& i) {
    std::vector<std::pair<int, int>> out; /* outward (dimension, sign) */
    for (int j = 0; j < o.c.n; ++j) {
        if (face_velocity(o, shifted(i, j, +1), j) > 0.0) out.push_back({j, +1});
        if (face_velocity(o, i, j) < 0.0) out.push_back({j, -1});
    }
    std::vector<Idx> d;
    for (auto& a : out) d.push_back(shifted(i, a.first, a.second));
    for (size_t a = 0; a < out.size(); ++a)
        for (size_t b = a + 1; b < out.size(); ++b)
            if (out[a].first != out[b].first)
                d.push_back(shifted(shifted(i, out[a].first, out[a].second), out[b].first, out[b].second));
    return d;
}

/* Grow: insert D(S) with p = 0, S = {p > thr_rel max p}. The downwind sets
 * are found in parallel; the cells missing from the grid are inserted in the
 * order of the significant cells that name them. */
void grow(Oracle& o) {
    double pstar = o.c.thr_rel * max_p(o.P);
    const auto cells = cell_list(o.P);
    const int64_t N = (int64_t)cells.size();
    std::vector<std::vector<Idx>> add(N);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < N; ++i)
        if (cells[i]->second > pstar)
            for (auto& d : downwind(o, cells[i]->first))
                if (!o.P.count(d)) add[i].push_back(d);
    for (int64_t i = 0; i < N; ++i)
        for (auto& d : add[i]) o.P.emplace(d, 0.0);
}

/* Prune (Algorithm 3 with the directional rule of Sec. 3.3): keep S u D(S). */
void prune(Oracle& o) {
    double pstar = o.c.thr_rel * max_p(o.P);
    const auto cells = cell_list(o.P);
    const int64_t N = (int64_t)cells.size();
    std::vector<std::vector<Idx>> down(N);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < N; ++i)
        if (cells[i]->second > pstar) down[i] = downwind(o, cells[i]->first);
    std::unordered_set<Idx, IdxHash> keep;
    for (int64_t i = 0; i < N; ++i)
        if (cells[i]->second > pstar) {
            keep.insert(cells[i]->first);
            for (auto& d : down[i]) keep.insert(d);
        }
    for (auto it = o.P.begin(); it != o.P.end();) {
        if (keep.count(it->first)) ++it;
        else it = o.P.erase(it);
    }
}

/* CFL rate of a cell: sum_j |f_{i-e_j/2, j}| / h_j (Eq. 8 with |f|). */
double cfl_rate(const Oracle& o, const Idx& i) {
    double r = 0.0;
    for (int j = 0; j < o.c.n; ++j) r += std::fabs(face_velocity(o, i, j)) / o.c.h[j];
    return r;
}

/* max_i of the CFL rates over the grid (order-free). */
double max_rate(const Oracle& o) {
    const auto cells = cell_list(o.P);
    const int64_t N = (int64_t)cells.size();
    double r = 0.0;
#pragma omp parallel for reduction(max : r) schedule(static)
    for (int64_t i = 0; i < N; ++i) r = std::max(r, cfl_rate(o, cells[i]->first));
    return r;
}

double limiter(int kind, double theta) {
    if (kind == LIM_NONE) return 0.0;
    if (kind == LIM_LW) return 1.0;
    return std::max(0.0, std::min(std::min((1.0 + theta) / 2.0, 2.0), 2.0 * theta)); /* MC */
}

/* The faces of one dimension j that touch an active cell: the lower j-face of
 * every active cell X and of X + e_j, numbered in order of first appearance,
 * with the velocity through each face, the jump of P across it and the flux
 * being assembled. */
struct FaceSet {
    std::vector<Idx> X;                           /* face k is the lower j-face of cell X[k] */
    std::unordered_map<Idx, int64_t, IdxHash> at; /* X[k] -> k */
    std::vector<double> u, W, F;                  /* f_j on the face, P_X - P_{X-e_j}, flux */
    int64_t find(const Idx& Y) const {
        auto it = at.find(Y);
        return it == at.end() ? -1 : it->second;
    }
};

/* One DCU + CTU + high-resolution update of every active cell with time step
 * dt (Eq. 7, Algorithm 1, Sec. 2.1). Returns the new values of the active
 * cells; nothing is normalised. */
Field ctu_update(const Oracle& o, const Field& P, double dt) {
    const int n = o.c.n;
    const double* h = o.c.h;
    const auto cells = cell_list(P);
    const int64_t N = (int64_t)cells.size();
    std::vector<FaceSet> fs(n);
#pragma omp parallel for schedule(static, 1)
    for (int j = 0; j < n; ++j) {
        FaceSet& f = fs[j];
        f.at.reserve(2 * N);
        for (int64_t i = 0; i < N; ++i)
            for (int s = 0; s < 2; ++s) {
                Idx X = shifted(cells[i]->first, j, s);
                if (f.at.emplace(X, (int64_t)f.X.size()).second) f.X.push_back(X);
            }
        f.u.resize(f.X.size());
        f.W.resize(f.X.size());
        f.F.resize(f.X.size());
    }
    /* Eq. 7: donor cell upwind, with the face velocity and the jump kept */
    for (int j = 0; j < n; ++j) {
        FaceSet& f = fs[j];
        const int64_t M = (int64_t)f.X.size();
#pragma omp parallel for schedule(static)
        for (int64_t k = 0; k < M; ++k) {
            const Idx& X = f.X[k];
            const double u = face_velocity(o, X, j);
            const double Pl = get(P, shifted(X, j, -1)), Pr = get(P, X);
            f.u[k] = u;
            f.W[k] = Pr - Pl;
            f.F[k] = std::max(u, 0.0) * Pl + std::min(u, 0.0) * Pr;
        }
    }
    /* Algorithm 1, restated per wave: the jump W across the lower j-face of X
     * crosses that face in the direction of its velocity u, into the cell Y = X
     * (u > 0) or Y = X - e_j (u < 0). Inside Y the transverse velocity of
     * dimension l != j carries it on, through the upper l-face of Y where the
     * velocity there is positive and through the lower l-face of Y where it is
     * negative; each such flux loses u v dt / (2 h_j) W. One thread owns the
     * flux array of each dimension l and adds the waves in the order of the
     * emitting faces (j, then k). */
#pragma omp parallel for schedule(static, 1)
    for (int l = 0; l < n; ++l) {
        FaceSet& T = fs[l];
        for (int j = 0; j < n; ++j) {
            if (j == l) continue;
            const FaceSet& f = fs[j];
            for (size_t k = 0; k < f.X.size(); ++k) {
                const double u = f.u[k];
                if (u == 0.0) continue;
                const Idx Y = u > 0.0 ? f.X[k] : shifted(f.X[k], j, -1);
                const double Fstar = dt / (2.0 * h[j]) * f.W[k];
                const Idx Yup = shifted(Y, l, +1);
                const int64_t a = T.find(Yup), b = T.find(Y);
                if (a >= 0) T.F[a] -= u * std::max(face_velocity(o, Yup, l), 0.0) * Fstar;
                if (b >= 0) T.F[b] -= u * std::min(face_velocity(o, Y, l), 0.0) * Fstar;
            }
        }
    }
    /* High-resolution correction with a limited wave */
    if (o.c.limiter != LIM_NONE)
        for (int j = 0; j < n; ++j) {
            FaceSet& f = fs[j];
            const int64_t M = (int64_t)f.X.size();
#pragma omp parallel for schedule(static)
            for (int64_t k = 0; k < M; ++k) {
                const Idx& X = f.X[k];
                double W = f.W[k];
                if (W == 0.0) continue;
                double u = f.u[k];
                double Wup = u > 0.0 ? get(P, shifted(X, j, -1)) - get(P, shifted(X, j, -2))
                                     : get(P, shifted(X, j, +1)) - get(P, X);
                double theta = Wup / W;
                double au = std::fabs(u);
                f.F[k] += 0.5 * au * (1.0 - dt * au / h[j]) * limiter(o.c.limiter, theta) * W;
            }
        }
    /* conservative update of the active cells */
    std::vector<double> val(N);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        const Idx& X = cells[i]->first;
        double acc = 0.0;
        for (int j = 0; j < n; ++j)
            acc += dt / h[j] * (fs[j].F[fs[j].find(shifted(X, j, +1))] - fs[j].F[fs[j].find(X)]);
        val[i] = cells[i]->second - acc;
    }
    Field out;
    out.reserve(P.size());
    for (int64_t i = 0; i < N; ++i) out.emplace(cells[i]->first, val[i]);
    return out;
}

/* Exact sum of the stored values (per-thread partial sums, merged exactly). */
ExactSum exact_total(const Field& P) {
    const auto cells = cell_list(P);
    const int64_t N = (int64_t)cells.size();
    ExactSum total;
#pragma omp parallel
    {
        ExactSum part;
#pragma omp for schedule(static)
        for (int64_t i = 0; i < N; ++i) part.add(cells[i]->second);
#pragma omp critical
        total.merge(part);
    }
    return total;
}

/* (prod h) * sum p, summed exactly */
double mass(const Oracle& o) { return o.prod_h * exact_total(o.P).value(); }

/* p <- p / ((prod h) sum p) */
int normalise(Oracle& o) {
    double w = mass(o);
    if (!(w > 0.0) || !std::isfinite(w)) {
        o.err = "degenerate: total probability is not positive";
        return ORC_EDEGENERATE;
    }
    const auto cells = cell_list(o.P);
    const int64_t N = (int64_t)cells.size();
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) cells[i]->second = cells[i]->second / w;
    return ORC_OK;
}

/* Solve for the inverse of a small symmetric positive definite matrix by
 * Gauss-Jordan elimination with partial pivoting. Returns false if singular. */
bool invert(int m, const double* A, double* Ainv) {
    double a[6][12];
    for (int r = 0; r < m; ++r)
        for (int q = 0; q < 2 * m; ++q) a[r][q] = q < m ? A[r * m + q] : (q - m == r ? 1.0 : 0.0);
    for (int col = 0; col < m; ++col) {
        int piv = col;
        for (int r = col + 1; r < m; ++r)
            if (std::fabs(a[r][col]) > std::fabs(a[piv][col])) piv = r;
        if (a[piv][col] == 0.0) return false;
        if (piv != col)
            for (int q = 0; q < 2 * m; ++q) std::swap(a[piv][q], a[col][q]);
        double d = a[col][col];
        for (int q = 0; q < 2 * m; ++q) a[col][q] /= d;
        for (int r = 0; r < m; ++r) {
            if (r == col) continue;
            double f = a[r][col];
            for (int q = 0; q < 2 * m; ++q) a[r][q] -= f * a[col][q];
        }
    }
    for (int r = 0; r < m; ++r)
        for (int q = 0; q < m; ++q) Ainv[r * m + q] = a[r][m + q];
    return true;
}

int one_step(Oracle& o, double t_target, int64_t* updates) {
    grow(o);
    double rmax = max_rate(o);
    double remaining = t_target - o.t;
    double dt = rmax > 0.0 ? o.c.cfl / rmax : INFINITY;
    double t_new;
    if (dt >= remaining) { dt = remaining; t_new = t_target; }
    else t_new = o.t + dt;
    o.P = ctu_update(o, o.P, dt);
    *updates += (int64_t)o.P.size();
    o.t = t_new;
    o.last_dt = dt;
    o.step += 1;
    if (o.c.prune_interval > 0 && o.step % o.c.prune_interval == 0) prune(o);
    return normalise(o);
}

bool valid(const orc_config* c) {
    if (c->n < 1 || c->n > 6) return false;
    for (int j = 0; j < c->n; ++j)
        if (!(c->h[j] > 0.0)) return false;
    if (c->dynamics == DYN_LORENZ63 || c->dynamics == DYN_LORENZ63_SHIFTED) {
        if (c->n != 3) return false;
    }
    if (c->dynamics == DYN_LORENZ96 && c->n < 4) return false;
    if (c->dynamics < 0 || c->dynamics > 4) return false;
    if (c->limiter < 0 || c->limiter > 2) return false;
    if (!(c->cfl > 0.0) || !(c->thr_rel >= 0.0)) return false;
    return true;
}

bool key_less(const Idx& a, const Idx& b) { return a < b; }

}  // namespace

extern "C" {

void* orc_create(const orc_config* cfg) {
    if (!cfg || !valid(cfg)) return nullptr;
    Oracle* o = new Oracle;
    o->c = *cfg;
    o->prod_h = 1.0;
    for (int j = 0; j < cfg->n; ++j) o->prod_h *= cfg->h[j];
    return o;
}

void orc_destroy(void* h) { delete (Oracle*)h; }

const char* orc_last_error(void* h) { return ((Oracle*)h)->err.c_str(); }

/* Initial Gaussian N(mean, cov) sampled at cell centres, cells with
 * p > thr_rel * max p kept, then normalised. */
int orc_init_gaussian(void* h, const double* mean, const double* cov, double t0) {
    Oracle& o = *(Oracle*)h;
    const int n = o.c.n;
    double icov[36];
    if (!invert(n, cov, icov)) { o.err = "covariance is singular"; return ORC_EINVAL; }
    auto gauss = [&](const Idx& i) {
        double dx[6];
        for (int k = 0; k < n; ++k) dx[k] = centre(o, i, k) - mean[k];
        double q = 0.0;
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b) q += dx[a] * icov[a * n + b] * dx[b];
        return std::exp(-0.5 * q);
    };
    int ctr[6];
    for (int k = 0; k < n; ++k) ctr[k] = (int)std::lround((mean[k] - o.c.x0[k]) / o.c.h[k]);
    /* the box of half-width ceil(sqrt(r2 cov_kk) / h_k) + 1 around the mean's
     * cell, visited in lexicographic order (dimension 0 slowest) in chunks of
     * consecutive cells; visit(chunk, cell) */
    auto scan_box = [&](double r2, int64_t chunks, auto&& visit) {
        int lo[6];
        int64_t dims[6], total = 1;
        for (int k = 0; k < n; ++k) {
            int hw = (int)std::ceil(std::sqrt(r2 * cov[k * n + k]) / o.c.h[k]) + 1;
            lo[k] = ctr[k] - hw;
            dims[k] = 2 * (int64_t)hw + 1;
            total *= dims[k];
        }
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t c = 0; c < chunks; ++c) {
            const int64_t a = total * c / chunks, b = total * (c + 1) / chunks;
            for (int64_t lin = a; lin < b; ++lin) {
                Idx i{0, 0, 0, 0, 0, 0};
                int64_t r = lin;
                for (int k = n - 1; k >= 0; --k) {
                    i[k] = lo[k] + (int32_t)(r % dims[k]);
                    r /= dims[k];
                }
                visit(c, i);
            }
        }
    };
    double thr = o.c.thr_rel > 0.0 ? o.c.thr_rel : 1e-300;
    const int64_t chunks = 1024;
    std::vector<double> cmax(chunks, 0.0);
    scan_box(-2.0 * std::log(thr), chunks, [&](int64_t c, const Idx& i) { cmax[c] = std::max(cmax[c], gauss(i)); });
    double gmax = 0.0;
    for (double v : cmax) gmax = std::max(gmax, v);
    if (!(gmax > 0.0)) { o.err = "initial density underflows on the grid"; return ORC_EDEGENERATE; }
    double pstar = o.c.thr_rel * gmax;
    o.P.clear();
    std::vector<std::vector<std::pair<Idx, double>>> kept(chunks);
    scan_box(-2.0 * std::log(thr * gmax), chunks, [&](int64_t c, const Idx& i) {
        double g = gauss(i);
        if (g > pstar) kept[c].push_back({i, g});
    });
    for (auto& part : kept)
        for (auto& kv : part) o.P[kv.first] = kv.second;
    o.t = t0;
    o.step = 0;
    return normalise(o);
}

/* Load an explicit cell set; p is taken as given (not renormalised); step0
 * steps are counted as already taken (the prune schedule continues from it). */
int orc_init_cells(void* h, const int32_t* idx, const double* p, int64_t N, double t0, int64_t step0) {
    Oracle& o = *(Oracle*)h;
    o.P.clear();
    for (int64_t c = 0; c < N; ++c) {
        Idx i{0, 0, 0, 0, 0, 0};
        for (int k = 0; k < o.c.n; ++k) i[k] = idx[c * o.c.n + k];
        o.P[i] = p[c];
    }
    o.t = t0;
    o.step = step0;
    return ORC_OK;
}

/* Propagate until t == t_end: steps of grow, dt (Eq. 8), flux update, prune
 * (when due) and normalisation, without measurements. */
int orc_propagate_steps(void* h, double t_end, int64_t max_steps, orc_stats* st);
int orc_propagate(void* h, double t_end, orc_stats* st) { return orc_propagate_steps(h, t_end, -1, st); }

/* The same, but at most max_steps steps (max_steps < 0: no cap). */
int orc_propagate_steps(void* h, double t_end, int64_t max_steps, orc_stats* st) {
    Oracle& o = *(Oracle*)h;
    int64_t steps = 0, updates = 0;
    int rc = ORC_OK;
    while (o.t < t_end && (max_steps < 0 || steps < max_steps)) {
        rc = one_step(o, t_end, &updates);
        ++steps;
        if (rc) break;
    }
    if (st) {
        st->steps = steps;
        st->cell_updates = updates;
        st->t = o.t;
        st->last_dt = o.last_dt;
        st->total_steps = o.step;
    }
    return rc;
}

/* Bayesian update with a Gaussian likelihood of the measurement y of the state
 * components H_idx[0..m) with covariance R (Eq. 4), then prune and normalise
 * (the constant C of Eq. 4 is the integral over the kept cells). */
int orc_correct_gaussian(void* h, const double* y, const double* R, const int32_t* H_idx, int32_t m) {
    Oracle& o = *(Oracle*)h;
    double Rinv[36];
    if (m < 1 || m > 6 || !invert(m, R, Rinv)) { o.err = "bad measurement"; return ORC_EINVAL; }
    for (int a = 0; a < m; ++a)
        if (H_idx[a] < 0 || H_idx[a] >= o.c.n) { o.err = "bad measurement index"; return ORC_EINVAL; }
    const auto cells = cell_list(o.P);
    const int64_t N = (int64_t)cells.size();
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        auto& kv = *cells[i];
        double r[6];
        for (int a = 0; a < m; ++a) r[a] = y[a] - centre(o, kv.first, H_idx[a]);
        double q = 0.0;
        for (int a = 0; a < m; ++a)
            for (int b = 0; b < m; ++b) q += r[a] * Rinv[a * m + b] * r[b];
        kv.second = std::exp(-0.5 * q) * kv.second;
    }
    prune(o);
    return normalise(o);
}

int64_t orc_count(void* h) { return (int64_t)((Oracle*)h)->P.size(); }

/* Cells in lexicographic key order (dimension 0 slowest). */
int64_t orc_read_cells(void* h, int32_t* idx, double* p, int64_t cap) {
    Oracle& o = *(Oracle*)h;
    std::vector<Idx> keys;
    keys.reserve(o.P.size());
    for (auto& kv : o.P) keys.push_back(kv.first);
    std::sort(keys.begin(), keys.end(), key_less);
    int64_t N = (int64_t)keys.size();
    for (int64_t c = 0; c < N && c < cap; ++c) {
        for (int k = 0; k < o.c.n; ++k) idx[c * o.c.n + k] = keys[c][k];
        p[c] = o.P[keys[c]];
    }
    return N;
}

/* mean = (prod h) sum x p ; cov = (prod h) sum (x-mean)(x-mean)^T p */
void orc_moments(void* h, double* mean, double* cov) {
    Oracle& o = *(Oracle*)h;
    const int n = o.c.n;
    const auto cells = cell_list(o.P);
    const int64_t N = (int64_t)cells.size();
    /* sum over the cells of term(cell), exactly, for each of `count` terms */
    auto exact = [&](int count, auto&& term, double* out) {
        std::vector<ExactSum> tot(count);
#pragma omp parallel
        {
            std::vector<ExactSum> part(count);
#pragma omp for schedule(static)
            for (int64_t i = 0; i < N; ++i)
                for (int q = 0; q < count; ++q) part[q].add(term(*cells[i], q));
#pragma omp critical
            for (int q = 0; q < count; ++q) tot[q].merge(part[q]);
        }
        for (int q = 0; q < count; ++q) out[q] = o.prod_h * tot[q].value();
    };
    exact(n, [&](const std::pair<const Idx, double>& kv, int a) { return centre(o, kv.first, a) * kv.second; },
          mean);
    exact(n * n,
          [&](const std::pair<const Idx, double>& kv, int q) {
              const int a = q / n, b = q % n;
              return (centre(o, kv.first, a) - mean[a]) * (centre(o, kv.first, b) - mean[b]) * kv.second;
          },
          cov);
}

/* ---- single pieces of the step, for the pins in tests/ ---- */

/* One DCU/CTU/HR update with a given dt on the current set; no grow, no
 * prune, no normalisation, time unchanged. */
int orc_ctu_step(void* h, double dt) {
    Oracle& o = *(Oracle*)h;
    o.P = ctu_update(o, o.P, dt);
    return ORC_OK;
}

int orc_grow(void* h) { grow(*(Oracle*)h); return ORC_OK; }
int orc_prune(void* h) { prune(*(Oracle*)h); return ORC_OK; }
int orc_normalise(void* h) { return normalise(*(Oracle*)h); }

/* dt the next step would take towards t_target (after its grow). */
double orc_cfl_dt(void* h) {
    Oracle& o = *(Oracle*)h;
    double rmax = max_rate(o);
    return rmax > 0.0 ? o.c.cfl / rmax : INFINITY;
}

/* Drift f_j(x) of the configured model at an arbitrary point. */
double orc_drift(void* h, const double* x, int32_t j) { return drift(((Oracle*)h)->c, x, j); }

/* Face velocity f_{X - e_j/2, j} at cell X. */
double orc_face_velocity(void* h, const int32_t* X, int32_t j) {
    Oracle& o = *(Oracle*)h;
    Idx i{0, 0, 0, 0, 0, 0};
    for (int k = 0; k < o.c.n; ++k) i[k] = X[k];
    return face_velocity(o, i, j);
}

/* Downwind set of cell X; returns its size and writes up to cap cells. */
int32_t orc_downwind(void* h, const int32_t* X, int32_t* out, int32_t cap) {
    Oracle& o = *(Oracle*)h;
    Idx i{0, 0, 0, 0, 0, 0};
    for (int k = 0; k < o.c.n; ++k) i[k] = X[k];
    auto d = downwind(o, i);
    for (int32_t q = 0; q < (int32_t)d.size() && q < cap; ++q)
        for (int k = 0; k < o.c.n; ++k) out[q * o.c.n + k] = d[q][k];
    return (int32_t)d.size();
}

/* Exact sum of m doubles, correctly rounded. */
double orc_exact_sum(const double* x, int64_t m) {
    ExactSum s;
    for (int64_t q = 0; q < m; ++q) s.add(x[q]);
    return s.value();
}

/* The one-step update of chosen cells alone, computed from the current state
 * after a grow: for each chosen cell, Algorithm 1 and the corrections run on
 * the active cells of its stencil (the cells whose values can reach it in one
 * step), and the value at the cell is returned. No state changes. */
int orc_ctu_sample(void* h, double dt, const int32_t* idx, int64_t m, double* out) {
    Oracle& o = *(Oracle*)h;
    const int n = o.c.n;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < m; ++q) {
        Idx i{0, 0, 0, 0, 0, 0};
        for (int k = 0; k < n; ++k) i[k] = idx[q * n + k];
        if (!o.P.count(i)) { out[q] = NAN; continue; }
        std::vector<Idx> st{i};
        for (int j = 0; j < n; ++j)
            for (int s : {-2, -1, 1, 2}) st.push_back(shifted(i, j, s));
        for (int j = 0; j < n; ++j)
            for (int l = j + 1; l < n; ++l)
                for (int s : {-1, 1})
                    for (int r : {-1, 1}) st.push_back(shifted(shifted(i, j, s), l, r));
        Field sub;
        for (auto& x : st) {
            auto it = o.P.find(x);
            if (it != o.P.end()) sub.emplace(x, it->second);
        }
        Field res = ctu_update(o, sub, dt);
        out[q] = res[i];
    }
    return ORC_OK;
}

/* Threads of the parallel loops (0: the OpenMP default); returns the number
 * in use afterwards (1 in a build without OpenMP). Results do not depend on it. */
int32_t orc_set_threads(int32_t k) {
#ifdef _OPENMP
    if (k > 0) omp_set_num_threads(k);
    return (int32_t)omp_get_max_threads();
#else
    (void)k;
    return 1;
#endif
}

double orc_time(void* h) { return ((Oracle*)h)->t; }
int64_t orc_steps(void* h) { return ((Oracle*)h)->step; }

}  /* extern "C" */
