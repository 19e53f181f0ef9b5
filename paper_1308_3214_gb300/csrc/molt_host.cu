// molt_host.cu -- host-side constants of the scheme shared by the single
// problem and the batched entry points: the update weights and beta_max
// (Sec. 3), the expansion of F in the per-axis D_gamma (Sec. 4), and the
// per-axis constants of the difference form of D.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <string>
#include <vector>

#include "molt_internal.h"

namespace molt {

// ---------------------------------------------------------------------------
// Scheme coefficients (Sec. 3, eq. update_P; Sec. 4, eq. Full_2D)
// ---------------------------------------------------------------------------
static double binomial(int n, int k)
{
    if (k < 0 || k > n) return 0.0;
    double r = 1.0;
    for (int i = 0; i < k; ++i) r = r * (double)(n - i) / (double)(i + 1);
    return r;
}

// weight of C^m D^{p-m}: (-1)^m 2 beta^{2m}/(2m)! binom(p-1, m-1)
double term_weight(int p, int m, double beta)
{
    double f = 1.0;
    for (int i = 2; i <= 2 * m; ++i) f *= i;
    double sgn = (m % 2) ? -1.0 : 1.0;
    return sgn * 2.0 * std::pow(beta, 2.0 * m) / f * binomial(p - 1, m - 1);
}

static double stability_sum(int P, double beta)   // S(beta, 1) = -sum_p A_p(beta)
{
    double s = 0.0;
    for (int p = 1; p <= P; ++p)
        for (int m = 1; m <= p; ++m) s -= term_weight(p, m, beta);
    return s;
}

double beta_max_of(int P)
{
    if (P < 1 || P > kMaxP) return -1.0;
    double prev = 0.0;
    for (int i = 1; i <= 4000; ++i) {
        double b = 1e-3 * i;
        if (stability_sum(P, b) >= 4.0) {
            double lo = prev, hi = b;
            for (int it = 0; it < 100; ++it) {
                double mid = 0.5 * (lo + hi);
                (stability_sum(P, mid) >= 4.0 ? hi : lo) = mid;
            }
            return 0.5 * (lo + hi);
        }
        prev = b;
    }
    return -1.0;
}

// Dense polynomial in up to three commuting variables D_x, D_y, D_z with
// degree <= deg in each.
struct Poly {
    int nv, deg;
    std::vector<double> c;
    Poly(int nv_, int deg_) : nv(nv_), deg(deg_), c((size_t)std::pow(deg_ + 1, nv_), 0.0) {}
    int idx(int i, int j, int k) const { return i + (deg + 1) * (j + (deg + 1) * k); }
    static Poly one(int nv, int deg) { Poly p(nv, deg); p.c[0] = 1.0; return p; }
    static Poly var(int nv, int deg, int a)
    {
        Poly p(nv, deg);
        int e[3] = {0, 0, 0};
        e[a] = 1;
        p.c[p.idx(e[0], e[1], e[2])] = 1.0;
        return p;
    }
};

static Poly padd(const Poly &a, const Poly &b, double sb = 1.0)
{
    Poly r = a;
    for (size_t i = 0; i < r.c.size(); ++i) r.c[i] += sb * b.c[i];
    return r;
}

static bool pmul(const Poly &a, const Poly &b, Poly &r)
{
    r = Poly(a.nv, a.deg);
    const int D = a.deg, K = a.nv >= 3 ? D : 0, J = a.nv >= 2 ? D : 0;
    for (int k1 = 0; k1 <= K; ++k1) for (int j1 = 0; j1 <= J; ++j1) for (int i1 = 0; i1 <= D; ++i1) {
        double x = a.c[a.idx(i1, j1, k1)];
        if (x == 0.0) continue;
        for (int k2 = 0; k2 <= K; ++k2) for (int j2 = 0; j2 <= J; ++j2) for (int i2 = 0; i2 <= D; ++i2) {
            double y = b.c[b.idx(i2, j2, k2)];
            if (y == 0.0) continue;
            if (i1 + i2 > D || j1 + j2 > D || k1 + k2 > D) return false;
            r.c[r.idx(i1 + i2, j1 + j2, k1 + k2)] += x * y;
        }
    }
    return true;
}

// F = sum_p sum_m w_pm C^m D^{p-m} with C, D expressed through the per-axis
// D_gamma: L_gamma^{-1} = 1 - D_gamma (eq. LD_gam), so
//   C = sum_g D_g prod_{g' != g} (1 - D_g')   (eqs. C_def_ADI, C_def_ADI_3)
//   D = 1 - prod_g (1 - D_g)                  (eqs. D_def_ADI, D_def_ADI_3)
// (1D: C = D = D_x).  The per-axis operators act on different indices of a
// tensor grid and commute, so F is a polynomial of degree <= P in each D_g.
bool expand_coefficients(int ndim, int P, double beta, std::vector<double> &out)
{
    const int nv = ndim;
    Poly one = Poly::one(nv, P);
    std::vector<Poly> Dg, Lg;
    for (int a = 0; a < nv; ++a) {
        Dg.push_back(Poly::var(nv, P, a));
        Lg.push_back(padd(one, Dg.back(), -1.0));
    }
    Poly C(nv, P), Dop(nv, P), tmp(nv, P);
    Poly prodL = one;
    for (int a = 0; a < nv; ++a) { if (!pmul(prodL, Lg[a], tmp)) return false; prodL = tmp; }
    Dop = padd(one, prodL, -1.0);
    for (int g = 0; g < nv; ++g) {
        Poly t = Dg[g];
        for (int a = 0; a < nv; ++a) if (a != g) { if (!pmul(t, Lg[a], tmp)) return false; t = tmp; }
        C = padd(C, t);
    }
    Poly F(nv, P);
    std::vector<Poly> Cp(P + 1, one), Dp(P + 1, one);
    for (int k = 1; k <= P; ++k) {
        if (!pmul(Cp[k - 1], C, Cp[k])) return false;
        if (!pmul(Dp[k - 1], Dop, Dp[k])) return false;
    }
    for (int p = 1; p <= P; ++p)
        for (int m = 1; m <= p; ++m) {
            if (!pmul(Cp[m], Dp[p - m], tmp)) return false;
            F = padd(F, tmp, term_weight(p, m, beta));
        }
    out = F.c;
    return true;
}

// ---------------------------------------------------------------------------
// Per-axis constants of the difference form of D (see molt_kernels.cuh)
// ---------------------------------------------------------------------------
// R = (1 - d)/nu^2 - (1 + d)/(2 nu): weight of the second difference in an
// increment of the quadratic rule.  Series for small nu, where the two terms
// cancel: R = sum_{k>=3} (-1)^{k+1} (2 - k) nu^{k-2} / (2 k!).
double quad_R(double nu)
{
    if (nu < 0.25) {
        double s = 0.0, pw = nu, fact = 6.0;   // k = 3: nu^1, 3!
        for (int k = 3; k < 28; ++k) {
            double sign = ((k + 1) % 2 == 0) ? 1.0 : -1.0;
            s += sign * (2.0 - k) * pw / (2.0 * fact);
            pw *= nu;
            fact *= (k + 1);
        }
        return s;
    }
    double om = -std::expm1(-nu);          // 1 - d
    double d = std::exp(-nu);
    return (om - 0.5 * nu * (1.0 + d)) / (nu * nu);
}

void axis_constants(double nu, int64_t n, int bc, int quad, AxisDev &A)
{
    A.n = (int)n;
    A.m = (int)std::max<int64_t>(2, (n + 31) / 32);
    A.ms = (A.m % 2 == 0) ? A.m + 1 : A.m;
    A.mmagic = (unsigned)(((1ull << 32) + (unsigned long long)A.m - 1) / (unsigned long long)A.m);
    A.ls = 0;
    A.d = std::exp(-nu);
    const double khalf = -std::expm1(-2.0 * nu) / (2.0 * nu);   // K/2 = (1 - d^2)/(2 nu)
    const double R = (quad >= 2) ? quad_R(nu) : 0.0;
    A.c1 = -(khalf + R);
    A.c2 = 0.5 * R * A.d;
    if (bc == BC_PERIODIC) {
        A.mu = std::exp(-nu * (double)n);
        A.inv = -1.0 / std::expm1(-nu * (double)n);
    } else {
        A.mu = std::exp(-nu * (double)(n - 1));
        A.inv = -1.0 / std::expm1(-2.0 * nu * (double)(n - 1));
    }
    for (int k = 0; k < 5; ++k) A.dm[k] = std::exp(-nu * (double)A.m * (double)(1 << k));
    axis_mirror(A);
}

// ---------------------------------------------------------------------------
// History gradient by checkpoint-and-recompute (the adjoint of the forward
// map u^0 -> (u^0 .. u^N); see mol_adjoint_history in molt.h)
// ---------------------------------------------------------------------------
bool alloc_injected_failure();

mol_status history_gradient_run(const HistoryOps &o, const double *u0, int64_t N, int64_t K, mol_grad_fn fn,
                                void *user, double *grad, cudaStream_t s)
{
    if (N < 1 || K < 1 || !fn) return o.fail(o.ctx, MOL_EINVAL, "need nsteps >= 1, checkpoint_every >= 1, grad_fn");
    const int64_t nck = (N - 1) / K + 1;                   // checkpoints at c = 1 + i K <= N
    const int64_t seg = std::min<int64_t>(K, N);
    const size_t fb = sizeof(double) * (size_t)o.N;
    const size_t total = fb * (size_t)(2 * nck + seg + 4);
    double *buf = nullptr;
    if (alloc_injected_failure()) return o.fail(o.ctx, MOL_ENOMEM, "history workspace allocation failed (injected)");
    cudaError_t e = cudaMalloc(&buf, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return o.fail(o.ctx, MOL_ENOMEM, ("history workspace of " + std::to_string(total) + " bytes").c_str());
    }
    auto ck = [&](int64_t i, int which) { return buf + (size_t)(2 * i + which) * o.N; };
    double *states = buf + (size_t)(2 * nck) * o.N;
    double *mu[3] = {states + (size_t)seg * o.N, states + (size_t)(seg + 1) * o.N, states + (size_t)(seg + 2) * o.N};
    double *g = states + (size_t)(seg + 3) * o.N;
    mol_status st = MOL_OK;
    auto cuda_ok = [&](cudaError_t r, const char *what) {
        if (r == cudaSuccess) return true;
        st = o.fail(o.ctx, MOL_ECUDA, (std::string(what) + ": " + cudaGetErrorString(r)).c_str());
        return false;
    };
    // forward: (u^{c-1}, u^c) at every checkpoint
    if (cuda_ok(cudaMemcpyAsync(ck(0, 0), u0, fb, cudaMemcpyDeviceToDevice, s), "copy u0"))
        st = o.start(o.ctx, u0, ck(0, 1), s);
    for (int64_t i = 1; i < nck && st == MOL_OK; ++i) {
        if (!cuda_ok(cudaMemcpyAsync(ck(i, 0), ck(i - 1, 0), 2 * fb, cudaMemcpyDeviceToDevice, s), "copy checkpoint"))
            break;
        st = o.step(o.ctx, ck(i, 0), ck(i, 1), K, s);
    }
    // backward: recompute each segment's states, then run the adjoint through them
    int i0 = 0, i1 = 1, i2 = 2;                             // mu^n, mu^{n+1}, mu^{n+2}
    if (st == MOL_OK && cuda_ok(cudaMemsetAsync(mu[i1], 0, fb, s), "clear") &&
        cuda_ok(cudaMemsetAsync(mu[i2], 0, fb, s), "clear")) {
        for (int64_t i = nck - 1; i >= 0 && st == MOL_OK; --i) {
            const int64_t c = 1 + i * K, last = std::min(c + K - 1, N), m = last - c;
            if (!cuda_ok(cudaMemcpyAsync(states, ck(i, 1), fb, cudaMemcpyDeviceToDevice, s), "copy state")) break;
            if (m > 0 && (st = o.step_emit(o.ctx, ck(i, 0), ck(i, 1), m, states + o.N, s)) != MOL_OK) break;
            for (int64_t j = m; j >= 0 && st == MOL_OK; --j) {
                const int r = fn(c + j, states + (size_t)j * o.N, g, (void *)s, user);
                if (r != 0 && r != 1) { st = o.fail(o.ctx, MOL_EINVAL, "grad_fn returned an error"); break; }
                st = o.update_T(o.ctx, mu[i1], mu[i2], mu[i0], 2.0, -1.0, 1.0, r == 0 ? g : nullptr, s);
                const int t = i2; i2 = i1; i1 = i0; i0 = t;
            }
        }
    }
    if (st == MOL_OK) {
        const int r = fn(0, u0, g, (void *)s, user);
        if (r != 0 && r != 1) st = o.fail(o.ctx, MOL_EINVAL, "grad_fn returned an error");
        else st = o.update_T(o.ctx, mu[i1], mu[i2], grad, 1.0, -1.0, 0.5, r == 0 ? g : nullptr, s);
    }
    if (st == MOL_OK) cuda_ok(cudaStreamSynchronize(s), "stream synchronize");
    else cudaStreamSynchronize(s);
    cudaFree(buf);
    return st;
}

// ---------------------------------------------------------------------------
// Test hooks (host only): injected allocation failure, unstable beta
// ---------------------------------------------------------------------------
static std::atomic<long long> g_alloc_budget{-1};
static std::atomic<int> g_allow_unstable{0};

bool alloc_injected_failure()
{
    long long b = g_alloc_budget.load();
    while (b >= 0) {
        if (b == 0) return true;
        if (g_alloc_budget.compare_exchange_weak(b, b - 1)) return false;
    }
    return false;
}

bool unstable_allowed() { return g_allow_unstable.load() != 0; }

}  // namespace molt

extern "C" void mol_debug_fail_alloc(int64_t after) { molt::g_alloc_budget.store(after < 0 ? -1 : (long long)after); }
extern "C" void mol_debug_allow_unstable(int on) { molt::g_allow_unstable.store(on ? 1 : 0); }
