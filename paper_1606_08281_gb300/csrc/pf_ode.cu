// Deterministic likelihood of the Egf-Ras-Raf-Mek-Erk model (the paper's
// ODE example, Supp. "Egf-Ras-Raf-Mek-Erk model": reaction equations, species
// table, FRET noise model).  In a deterministic model the likelihood needs no
// particle filter: solve the ODE for theta and score the trajectory under the
// observation model (Sec. "A realistic example").
//
// GB300 layout: one thread per (theta row, input pattern), many per SM; each
// integrates the 14 concentrations with the explicit Dormand-Prince 5(4)
// pair (Dormand & Prince, J. Comput. Appl. Math. 6, 1980; FSAL, step control
// as in Hairer, Norsett & Wanner, "Solving ODEs I", Sec. II.4), stepping
// exactly onto every input switch time (the right-hand side jumps there) and
// every observation time, where it adds log N(y; R(x), sigma^2) with the
// FRET ratio R.  Stage vectors live in the thread's local memory (L1).  The
// work is FP64 arithmetic: per step six right-hand-side evaluations (with
// their Michaelis-Menten quotients) and the stage combinations.  A trajectory
// that needs more than max_steps steps (a stiff or diverging theta for an
// explicit method) stops with PF_ST_BUDGET and log-likelihood -inf, as the
// SSA does with its event budget.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "pf1606.h"
#include "pf_internal.h"

namespace pf {
namespace {

constexpr int kNs = 14;                  // states
constexpr int kThreads = 64;
constexpr double kThalf = 90.0;          // T_dusp = T_DUSP (min)

struct OdeArgs {
    const double *thetas;      // [M][36]
    const double *sw_t;        // switch times, all patterns
    const double *sw_v;        // switch values
    const int32_t *sw_off;     // [n_patterns + 1]
    const double *obs;         // [K]
    const double *y;           // [n_patterns][K]
    int64_t M;
    int32_t NP, K;
    double rtol, atol;
    int32_t max_steps;
    double *ll_f;              // [M * NP]
    uint8_t *st_f;             // [M * NP]
    uint32_t *steps_f;         // [M * NP] or null
};

// Right-hand side of the reaction equations; th = theta, u = egf input.
__device__ __forceinline__ void erk_rhs(const double *x, const double *th, double u, double *dx) {
    const double EGFR = x[0], EGFRa = x[1], Ras = x[2], Rasa = x[3], Raf = x[4], Rafa = x[5];
    const double MEK = x[6], MEKa = x[7], ERK = x[8], ERKa = x[9], NFB = x[10], NFBa = x[11];
    const double dusp = x[12], DUSP = x[13];
    const double v1 = th[0] * u * EGFR - th[1] * EGFRa;
    const double v2 = th[2] * EGFRa * Ras / (th[3] + Ras) - th[4] * Rasa / (th[5] + Rasa);
    const double kn2 = th[8] * th[8];
    const double v3 = th[6] * Rasa * Raf / (th[7] + Raf) * kn2 / (kn2 + NFBa * NFBa) -
                      th[9] * Rafa / (th[10] + Rafa);
    const double v4 = th[11] * Rafa * MEK / (th[12] + MEK) - th[13] * MEKa / (th[14] + MEKa);
    const double v5 = th[15] * MEKa * ERK / (th[16] + ERK) - th[17] * DUSP * ERKa / (th[18] + ERKa);
    const double e2 = EGFRa * EGFRa;
    const double v6 = th[19] * ERKa * NFB / (th[20] + NFB) * e2 / (th[21] * th[21] + e2) -
                      th[22] * NFBa / (th[23] + NFBa);
    const double a = 0.30102999566398119521 / kThalf;      // log10(2) / T, as printed
    const double ea2 = ERKa * ERKa;
    dx[0] = -v1; dx[1] = v1; dx[2] = -v2; dx[3] = v2; dx[4] = -v3; dx[5] = v3;
    dx[6] = -v4; dx[7] = v4; dx[8] = -v5; dx[9] = v5; dx[10] = -v6; dx[11] = v6;
    dx[12] = th[24] * (1.0 + th[25] * ea2 / (th[26] + ea2)) * a - dusp * a;
    dx[13] = dusp * a - DUSP * a;
}

__device__ __forceinline__ double fret(const double *x, const double *th) {
    const double ERK = x[8], ERKa = x[9], E = th[33];
    return th[31] * (ERKa * E * th[34] / ((ERK + (1.0 - E) * ERKa) * th[35]) + th[30]);
}

// Dormand-Prince 5(4) tableau.
constexpr double A21 = 1.0 / 5.0;
constexpr double A31 = 3.0 / 40.0, A32 = 9.0 / 40.0;
constexpr double A41 = 44.0 / 45.0, A42 = -56.0 / 15.0, A43 = 32.0 / 9.0;
constexpr double A51 = 19372.0 / 6561.0, A52 = -25360.0 / 2187.0, A53 = 64448.0 / 6561.0,
                 A54 = -212.0 / 729.0;
constexpr double A61 = 9017.0 / 3168.0, A62 = -355.0 / 33.0, A63 = 46732.0 / 5247.0,
                 A64 = 49.0 / 176.0, A65 = -5103.0 / 18656.0;
constexpr double B1 = 35.0 / 384.0, B3 = 500.0 / 1113.0, B4 = 125.0 / 192.0,
                 B5 = -2187.0 / 6784.0, B6 = 11.0 / 84.0;
constexpr double E1 = 71.0 / 57600.0, E3 = -71.0 / 16695.0, E4 = 71.0 / 1920.0,
                 E5 = -17253.0 / 339200.0, E6 = 22.0 / 525.0, E7 = -1.0 / 40.0;

__global__ void __launch_bounds__(kThreads) erk_kernel(const OdeArgs a) {
    // threads run pattern-major (g = p * M + m): the lanes of a warp share an
    // input pattern, so they stop at the same switch times and diverge less
    const int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= a.M * a.NP) return;
    const int p = static_cast<int>(g / a.M);
    const int64_t m = g - static_cast<int64_t>(p) * a.M;
    const int64_t f = m * a.NP + p;                 // result slot [m][p]
    double th[36];
    bool ok = true;
    for (int i = 0; i < 36; ++i) {
        th[i] = a.thetas[m * 36 + i];
        ok = ok && isfinite(th[i]) && th[i] > 0.0;
    }
    ok = ok && th[33] < 1.0;                         // FRET efficiency E in (0, 1)
    if (!ok) {
        a.ll_f[f] = __longlong_as_double(0x7FF8000000000000ll);
        a.st_f[f] = PF_ST_INVALID_THETA;
        if (a.steps_f) a.steps_f[f] = 0;
        return;
    }
    double x[kNs] = {th[27], 0.0, 0.1, 0.0, 0.7, 0.0, 0.68, 0.0, 0.26, 0.0, th[28], 0.0, th[29], th[29]};
    double k1[kNs], k2[kNs], k3[kNs], k4[kNs], k5[kNs], k6[kNs], k7[kNs], yt[kNs];
    const double *st = a.sw_t + a.sw_off[p];
    const int ns = a.sw_off[p + 1] - a.sw_off[p];
    const double *sv = a.sw_v + a.sw_off[p];
    const double *yp = a.y + static_cast<int64_t>(p) * a.K;
    const double sigma = th[32];
    const double lnorm = -log(sigma) - 0.91893853320467274178;    // -log sigma - log(2 pi)/2
    int si = 0;                                   // next switch index with st[si] > t
    while (si < ns && st[si] <= 0.0) ++si;
    double u = 0.0;
    for (int i = 0; i < ns && st[i] <= 0.0; ++i) u = sv[i];
    double t = 0.0, h = 1e-3, ll = 0.0;
    uint32_t steps = 0;
    int status = PF_ST_OK;
    bool fresh = true;                            // k1 must be evaluated
    for (int k = 0; k < a.K && status == PF_ST_OK; ++k) {
        const double tk = a.obs[k];
        while (t < tk && status == PF_ST_OK) {
            const double tstop = (si < ns && st[si] < tk) ? st[si] : tk;
            if (fresh) {
                erk_rhs(x, th, u, k1);
                fresh = false;
            }
            // one Dormand-Prince step, clipped to the stop
            bool last = false;
            double hh = h;
            if (t + hh >= tstop) {
                hh = tstop - t;
                last = true;
            }
            for (int i = 0; i < kNs; ++i) yt[i] = x[i] + hh * (A21 * k1[i]);
            erk_rhs(yt, th, u, k2);
            for (int i = 0; i < kNs; ++i) yt[i] = x[i] + hh * (A31 * k1[i] + A32 * k2[i]);
            erk_rhs(yt, th, u, k3);
            for (int i = 0; i < kNs; ++i) yt[i] = x[i] + hh * (A41 * k1[i] + A42 * k2[i] + A43 * k3[i]);
            erk_rhs(yt, th, u, k4);
            for (int i = 0; i < kNs; ++i)
                yt[i] = x[i] + hh * (A51 * k1[i] + A52 * k2[i] + A53 * k3[i] + A54 * k4[i]);
            erk_rhs(yt, th, u, k5);
            for (int i = 0; i < kNs; ++i)
                yt[i] = x[i] + hh * (A61 * k1[i] + A62 * k2[i] + A63 * k3[i] + A64 * k4[i] + A65 * k5[i]);
            erk_rhs(yt, th, u, k6);
            for (int i = 0; i < kNs; ++i)
                yt[i] = x[i] + hh * (B1 * k1[i] + B3 * k3[i] + B4 * k4[i] + B5 * k5[i] + B6 * k6[i]);
            erk_rhs(yt, th, u, k7);
            double err = 0.0;
            for (int i = 0; i < kNs; ++i) {
                const double ei = hh * (E1 * k1[i] + E3 * k3[i] + E4 * k4[i] + E5 * k5[i] + E6 * k6[i] +
                                        E7 * k7[i]);
                const double sc = a.atol + a.rtol * fmax(fabs(x[i]), fabs(yt[i]));
                const double r = ei / sc;
                err += r * r;
            }
            err = sqrt(err / kNs);
            if (!isfinite(err)) {
                status = PF_ST_NONFINITE;
                break;
            }
            if (++steps > static_cast<uint32_t>(a.max_steps)) {
                status = PF_ST_BUDGET;
                break;
            }
            if (err <= 1.0) {                         // accept
                t = last ? tstop : t + hh;
                for (int i = 0; i < kNs; ++i) {
                    x[i] = yt[i];
                    k1[i] = k7[i];                    // first same as last
                }
                const double fac = err > 0.0 ? fmin(5.0, fmax(0.2, 0.9 * pow(err, -0.2))) : 5.0;
                if (!last || hh * fac < h) h = hh * fac;
                if (last && si < ns && st[si] == tstop) {   // the input switches here
                    while (si < ns && st[si] <= tstop) u = sv[si++];
                    fresh = true;
                }
            } else {                                  // reject: shrink and retry
                h = hh * fmax(0.2, 0.9 * pow(err, -0.2));
            }
        }
        if (status != PF_ST_OK) break;
        const double R = fret(x, th);
        const double z = (yp[k] - R) / sigma;
        ll += lnorm - 0.5 * z * z;
    }
    a.ll_f[f] = status == PF_ST_OK ? ll : -INFINITY;
    a.st_f[f] = static_cast<uint8_t>(status);
    if (a.steps_f) a.steps_f[f] = steps;
}

__global__ void erk_reduce_kernel(const double *ll_f, const uint8_t *st_f, int64_t M, int NP,
                                  double *loglik, uint8_t *status) {
    const int64_t m = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double sum = 0.0;
    int st = PF_ST_OK;
    for (int p = 0; p < NP; ++p) {
        const int s = st_f[m * NP + p];
        if (st == PF_ST_OK && s != PF_ST_OK) st = s;
        sum += ll_f[m * NP + p];
    }
    double out = sum;
    if (st == PF_ST_INVALID_THETA) out = __longlong_as_double(0x7FF8000000000000ll);
    else if (st != PF_ST_OK) out = -INFINITY;
    loglik[m] = out;
    if (status) status[m] = static_cast<uint8_t>(st);
}

struct OBuf {
    void *p = nullptr;
    cudaStream_t s = nullptr;
    ~OBuf() { if (p) cudaFreeAsync(p, s); }
    cudaError_t alloc(size_t bytes, cudaStream_t st) {
        s = st;
        return bytes ? cudaMallocAsync(&p, bytes, st) : cudaSuccess;
    }
};

}  // namespace
}  // namespace pf

#define ODE_CUDA(call, what)                                          \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return pf::cuda_fail(e_, what);        \
    } while (0)

extern "C" int pf_erk_loglik(const double *thetas, int64_t M, const double *switch_times,
                             const double *switch_values, const int32_t *switch_offsets,
                             int32_t n_patterns, const double *obs_times, int32_t K,
                             const double *y, double *loglik, uint8_t *status,
                             const pf_ode_options *opt) {
    using pf::fail;
    pf::clear_error();
    pf_ode_options o{};
    if (opt) o = *opt;
    if (M < 0) return fail(PF_EINVAL, "M < 0");
    if (n_patterns < 1 || n_patterns > 1024) return fail(PF_EINVAL, "n_patterns %d outside 1..1024", n_patterns);
    if (K < 1 || K >= (1 << 20)) return fail(PF_EINVAL, "K %d outside 1..2^20-1", K);
    if (!switch_times || !switch_values || !switch_offsets || !obs_times)
        return fail(PF_EINVAL, "switch and observation arrays are required");
    if (M > 0 && (!thetas || !y || !loglik)) return fail(PF_EINVAL, "NULL array argument");
    if (M * (int64_t)n_patterns > 0x7FFFFFFFll) return fail(PF_EINVAL, "M * n_patterns must be < 2^31");
    int rc = pf::check_obs_times(obs_times, K);
    if (rc) return rc;
    if (!(obs_times[0] > 0.0)) return fail(PF_EINVAL, "obs_times[0] must be > 0 (the state at 0 is fixed)");
    if (switch_offsets[0] != 0) return fail(PF_EINVAL, "switch_offsets[0] must be 0");
    for (int p = 0; p < n_patterns; ++p) {
        if (switch_offsets[p + 1] < switch_offsets[p]) return fail(PF_EINVAL, "switch_offsets must not decrease");
        for (int i = switch_offsets[p]; i < switch_offsets[p + 1]; ++i) {
            if (!std::isfinite(switch_times[i]) || !std::isfinite(switch_values[i]) || switch_values[i] < 0.0)
                return fail(PF_EINVAL, "switch %d: times finite, values finite and >= 0", i);
            if (i > switch_offsets[p] && !(switch_times[i] > switch_times[i - 1]))
                return fail(PF_EINVAL, "switch times of pattern %d must increase", p);
        }
    }
    const double rtol = o.rtol > 0.0 ? o.rtol : 1e-10, atol = o.atol > 0.0 ? o.atol : 1e-13;
    if (!(rtol >= 1e-14 && rtol < 1.0) || !(atol > 0.0)) return fail(PF_EINVAL, "rtol in [1e-14, 1), atol > 0");
    const int max_steps = o.max_steps > 0 ? o.max_steps : 200000;
    if (M == 0) return PF_OK;

    cudaStream_t s = static_cast<cudaStream_t>(o.stream);
    const int NP = n_patterns, nsw = switch_offsets[NP];
    const int64_t F = M * NP;
    pf::OdeArgs a{};
    a.M = M; a.NP = NP; a.K = K; a.rtol = rtol; a.atol = atol; a.max_steps = max_steps;
    pf::OBuf b_sw, b_obs, b_th, b_y, b_ll, b_st, b_llf, b_stf, b_steps;
    // switch tables and observation times: one small host-to-device copy
    std::vector<unsigned char> tab(sizeof(double) * (2 * (size_t)nsw + K) + sizeof(int32_t) * (NP + 1));
    double *tt = reinterpret_cast<double *>(tab.data());
    std::copy(switch_times, switch_times + nsw, tt);
    std::copy(switch_values, switch_values + nsw, tt + nsw);
    std::copy(obs_times, obs_times + K, tt + 2 * nsw);
    std::copy(switch_offsets, switch_offsets + NP + 1, reinterpret_cast<int32_t *>(tt + 2 * nsw + K));
    ODE_CUDA(b_sw.alloc(tab.size(), s), "alloc tables");
    ODE_CUDA(cudaMemcpyAsync(b_sw.p, tab.data(), tab.size(), cudaMemcpyHostToDevice, s), "copy tables");
    const double *dt = static_cast<const double *>(b_sw.p);
    a.sw_t = dt;
    a.sw_v = dt + nsw;
    a.obs = dt + 2 * nsw;
    a.sw_off = reinterpret_cast<const int32_t *>(dt + 2 * nsw + K);
    double *d_ll = loglik;
    uint8_t *d_st = status;
    const size_t n_th = sizeof(double) * 36 * (size_t)M, n_y = sizeof(double) * (size_t)NP * K;
    if (o.device_ptrs) {
        a.thetas = thetas;
        a.y = y;
    } else {
        ODE_CUDA(b_th.alloc(n_th, s), "alloc thetas");
        ODE_CUDA(b_y.alloc(n_y, s), "alloc y");
        ODE_CUDA(b_ll.alloc(sizeof(double) * M, s), "alloc loglik");
        ODE_CUDA(b_st.alloc(M, s), "alloc status");
        ODE_CUDA(cudaMemcpyAsync(b_th.p, thetas, n_th, cudaMemcpyHostToDevice, s), "copy thetas");
        ODE_CUDA(cudaMemcpyAsync(b_y.p, y, n_y, cudaMemcpyHostToDevice, s), "copy y");
        a.thetas = static_cast<const double *>(b_th.p);
        a.y = static_cast<const double *>(b_y.p);
        d_ll = static_cast<double *>(b_ll.p);
        d_st = static_cast<uint8_t *>(b_st.p);
    }
    if (o.ll_pattern && o.device_ptrs) {
        a.ll_f = o.ll_pattern;
    } else {
        ODE_CUDA(b_llf.alloc(sizeof(double) * F, s), "alloc per-pattern values");
        a.ll_f = static_cast<double *>(b_llf.p);
    }
    ODE_CUDA(b_stf.alloc(F, s), "alloc per-pattern status");
    a.st_f = static_cast<uint8_t *>(b_stf.p);
    if (o.steps && o.device_ptrs) {
        a.steps_f = o.steps;
    } else if (o.steps) {
        ODE_CUDA(b_steps.alloc(sizeof(uint32_t) * F, s), "alloc steps");
        a.steps_f = static_cast<uint32_t *>(b_steps.p);
    }
    pf::erk_kernel<<<(unsigned)((F + pf::kThreads - 1) / pf::kThreads), pf::kThreads, 0, s>>>(a);
    ODE_CUDA(cudaGetLastError(), "ode launch");
    pf::erk_reduce_kernel<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(a.ll_f, a.st_f, M, NP, d_ll, d_st);
    ODE_CUDA(cudaGetLastError(), "ode reduce launch");
    if (!o.device_ptrs) {
        ODE_CUDA(cudaMemcpyAsync(loglik, d_ll, sizeof(double) * M, cudaMemcpyDeviceToHost, s), "copy loglik");
        if (status) ODE_CUDA(cudaMemcpyAsync(status, d_st, M, cudaMemcpyDeviceToHost, s), "copy status");
        if (o.ll_pattern) ODE_CUDA(cudaMemcpyAsync(o.ll_pattern, a.ll_f, sizeof(double) * F, cudaMemcpyDeviceToHost, s), "copy per-pattern values");
        if (o.steps) ODE_CUDA(cudaMemcpyAsync(o.steps, a.steps_f, sizeof(uint32_t) * F, cudaMemcpyDeviceToHost, s), "copy steps");
        ODE_CUDA(cudaStreamSynchronize(s), "synchronize");
    }
    return PF_OK;
}
