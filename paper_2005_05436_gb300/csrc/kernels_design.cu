// Design-side kernels: SIMP modulus (Eq. 5), cone-weight density filter and its
// chain rule (Eqs. 2, 7), Heaviside projection with the volume-preserving eta
// (Eqs. 1, 8, 15), the OC update with the lambda# bracket (Eqs. 13-14, 17), and
// the vector kernels of preconditioned CG.
#include "kernels.h"

namespace topo {

// ------------------------------------------------------------- modulus --

template <typename T>
__global__ void k_modulus(long long n, const double* __restrict__ x, double penal, double E0,
                          double Emin, T* __restrict__ E) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) E[i] = (T)(Emin + powp(x[i], penal) * (E0 - Emin));
}

template <typename T>
void launch_modulus(long long n, const double* x, double penal, double E0, double Emin, T* E,
                    cudaStream_t st) {
    k_modulus<T><<<div_up(n, 256), 256, 0, st>>>(n, x, penal, E0, Emin, E);
    TOPO_CHECK_LAUNCH();
}
template void launch_modulus<double>(long long, const double*, double, double, double, double*, cudaStream_t);
template void launch_modulus<float>(long long, const double*, double, double, double, float*, cudaStream_t);

// -------------------------------------------------------------- filter --

__global__ void __launch_bounds__(256) k_filter(Dims d, FilterTaps taps, int bcN, const double* __restrict__ rHs,
                                                double rHs_const, const double* __restrict__ in,
                                                const double* __restrict__ dprj, double* __restrict__ out,
                                                const int8_t* __restrict__ passive,
                                                const double* __restrict__ keep) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= d.nel) return;
    const int ey = (int)(e % d.nely);
    const long long t = e / d.nely;
    const int ez = (int)(t % d.nelz);
    const int ex = (int)(t / d.nelz);
    double s = 0.0;
    for (int k = 0; k < taps.nw; ++k) {
        int jx = ex + taps.off[3 * k], jy = ey + taps.off[3 * k + 1], jz = ez + taps.off[3 * k + 2];
        if (bcN) {
            jx = mirror_index(jx, d.nelx);
            jy = mirror_index(jy, d.nely);
            jz = mirror_index(jz, d.nelz);
        } else if (jx < 0 || jx >= d.nelx || jy < 0 || jy >= d.nely || jz < 0 || jz >= d.nelz) {
            continue;
        }
        const long long j = jy + (long long)d.nely * (jz + (long long)d.nelz * jx);
        double v = in[j];
        if (dprj) v = v * dprj[j] * (rHs ? rHs[j] : rHs_const);
        s += taps.w[k] * v;
    }
    if (!dprj) s = s * (rHs ? rHs[e] : rHs_const);
    if (passive && passive[e] != 0) s = keep[e];
    out[e] = s;
}

void launch_filter(const Dims& d, const FilterTaps& taps, char bc, const double* rHs, double rHs_const,
                   const double* in, const double* dprj, double* out, const int8_t* passive,
                   const double* keep, cudaStream_t st, bool float_float) {
    if (launch_filter_tiled(d, taps, bc, rHs, rHs_const, in, dprj, out, passive, keep, float_float, st)) return;
    k_filter<<<div_up(d.nel, 256), 256, 0, st>>>(d, taps, bc == 'N', rHs, rHs_const, in, dprj, out,
                                                 passive, keep);
    TOPO_CHECK_LAUNCH();
}

__global__ void k_recip(long long n, const double* __restrict__ in, double* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = 1.0 / in[i];
}

void launch_recip(long long n, const double* in, double* out, cudaStream_t st) {
    k_recip<<<div_up(n, 256), 256, 0, st>>>(n, in, out);
    TOPO_CHECK_LAUNCH();
}

// ---------------------------------------------------------- projection --

__device__ __forceinline__ double prj_d(double x, double tb_eta, double den, double beta, double eta) {
    return (tb_eta + tanh(beta * (x - eta))) / den;
}

constexpr int PNT = 256;

// Cooperative kernel: every block evaluates the same Newton sequence from the
// same (deterministically reduced) sums.
__global__ void __launch_bounds__(PNT) k_project(long long n, const double* __restrict__ xt,
                                                 double* __restrict__ xphys, double* __restrict__ dprj,
                                                 double beta, double eta0, double volfrac, int vp,
                                                 double tol, int maxit, long long deadline,
                                                 double* partials, GridBarrier* bar, ProjectOut* out) {
    const long long stride = (long long)gridDim.x * PNT;
    const long long i0 = (long long)blockIdx.x * PNT + threadIdx.x;
    const double nd = (double)n;
    double eta = eta0;
    int it = 0, parity = 0, status = 0;

    // mean(prj(xt, e)) - volfrac
    auto gfun = [&](double e, double& f) -> bool {
        const double tb = tanh(beta * e), den = tb + tanh(beta * (1.0 - e));
        double v[1] = {0.0}, tot[1];
        for (long long i = i0; i < n; i += stride) v[0] += prj_d(xt[i], tb, den, beta, e);
        if (!grid_totals<PNT, 1>(v, partials, parity, bar, deadline, tot)) return false;
        parity ^= 1;
        f = tot[0] / nd - volfrac;
        return true;
    };
    // mean(d prj / d eta) = mean(-beta sech^2(beta(x-eta)) sinh(beta x) sinh(beta(1-x)) / sinh(beta))
    auto dgfun = [&](double e, double& g) -> bool {
        const double sb = sinh(beta);
        double v[1] = {0.0}, tot[1];
        for (long long i = i0; i < n; i += stride) {
            const double x = xt[i];
            const double th = tanh(beta * (x - e));
            v[0] += -beta * (1.0 - th * th) * sinh(beta * x) * sinh(beta * (1.0 - x)) / sb;
        }
        if (!grid_totals<PNT, 1>(v, partials, parity, bar, deadline, tot)) return false;
        parity ^= 1;
        g = tot[0] / nd;
        return true;
    };

    if (vp) {
        double f;
        if (!gfun(eta, f)) return;
        while (fabs(f) > tol && it < maxit) {
            double g;
            if (!dgfun(eta, g)) return;
            eta = eta - f / g;
            ++it;
            if (!(eta >= 0.0 && eta <= 1.0)) break;
            if (!gfun(eta, f)) return;
        }
        if (!(fabs(f) <= tol && eta >= 0.0 && eta <= 1.0)) {
            double lo = 0.0, hi = 1.0;
            for (int k = 0; k < 200; ++k) {
                eta = 0.5 * (lo + hi);
                if (!gfun(eta, f)) return;
                if (fabs(f) <= tol || hi - lo <= 1e-16) break;
                if (f > 0.0)
                    lo = eta;
                else
                    hi = eta;
                ++it;
            }
            if (!(fabs(f) <= tol)) status = (int)TO_ENOTCONV;
        }
    }
    const double tb = tanh(beta * eta), den = tb + tanh(beta * (1.0 - eta));
    for (long long i = i0; i < n; i += stride) {
        const double x = xt[i];
        const double th = tanh(beta * (x - eta));
        xphys[i] = (tb + th) / den;
        dprj[i] = beta * (1.0 - th * th) / den;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        out->eta = eta;
        out->newton = it;
        out->status = status;
    }
}

int project_max_blocks() {
    int dev = 0, nsm = 0, per = 0;
    TOPO_CUDA(cudaGetDevice(&dev));
    TOPO_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    TOPO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_project, PNT, 0));
    return nsm * (per < 2 ? per : 2);
}

void launch_project(long long n, const double* xt, double* xphys, double* dprj, double beta,
                    double eta0, double volfrac, int vp, double tol, int maxit, long long deadline,
                    double* partials, GridBarrier* bar, ProjectOut* out, int nblocks, cudaStream_t st) {
    TOPO_CUDA(cudaMemsetAsync(bar, 0, sizeof(GridBarrier), st));
    void* args[] = {&n, &xt, &xphys, &dprj, &beta, &eta0, &volfrac, &vp, &tol, &maxit, &deadline,
                    &partials, &bar, &out};
    TOPO_CUDA(cudaLaunchCooperativeKernel((void*)k_project, dim3(nblocks), dim3(PNT), args, 0, st));
    count_launches(1);
}

// ------------------------------------------------------------------ OC --

constexpr int ONT = 256;
constexpr int OC_DEPTH = 4;                      // bisection levels per pass
constexpr int OC_NC = (1 << OC_DEPTH) - 1;       // candidates per pass

__global__ void __launch_bounds__(ONT) k_oc(long long n, double* __restrict__ x, const double* __restrict__ dc,
                                            const double* __restrict__ dV0, const int8_t* __restrict__ passive,
                                            long long nact, double move, double volfrac, double tol,
                                            int maxit, long long deadline, double* __restrict__ ocp,
                                            double* partials, GridBarrier* bar, OcOut* out) {
    const long long stride = (long long)gridDim.x * ONT;
    const long long i0 = (long long)blockIdx.x * ONT + threadIdx.x;
    const double nd = (double)n;
    int parity = 0;

    // ocP (Eq. 14 without lambda) and the constant passive volume
    double s2[2] = {0.0, 0.0}, t2[2];
    for (long long i = i0; i < n; i += stride) {
        const bool act = !passive || passive[i] == 0;
        if (act) {
            const double o = x[i] * sqrt(fmax(0.0, -dc[i] / dV0[i]));
            ocp[i] = o;
            s2[0] += o;
        } else {
            s2[1] += x[i];
        }
    }
    if (!grid_totals<ONT, 2>(s2, partials, parity, bar, deadline, t2)) return;
    parity ^= 1;
    const double pas_sum = t2[1];
    double l1 = 0.0, l2 = (t2[0] / (double)nact) / volfrac;
    double lmid = l2;
    int steps = 0, status = 0;

    auto newx = [&](long long i, double inv_lm) {
        const double xi = x[i];
        return fmax(fmax(fmin(fmin(ocp[i] * inv_lm, xi + move), 1.0), xi - move), 0.0);
    };

    if (l2 > 0.0) {
        // reading R6: grow the bracket while the volume at l2 is still too large
        for (int grow = 0; grow < 60; ++grow) {
            double v[1] = {0.0}, tot[1];
            const double inv = 1.0 / l2;
            for (long long i = i0; i < n; i += stride)
                if (!passive || passive[i] == 0) v[0] += newx(i, inv);
            if (!grid_totals<ONT, 1>(v, partials, parity, bar, deadline, tot)) return;
            parity ^= 1;
            if (!((tot[0] + pas_sum) / nd > volfrac)) break;
            l1 = l2;
            l2 = 2.0 * l2;
        }
        lmid = l2;
        // bisection, OC_DEPTH levels per pass: the complete tree of the next
        // midpoints is evaluated in one sweep and then walked exactly as the
        // sequential bisection would.
        while ((l2 - l1) / (l1 + l2) > tol && steps < maxit) {
            double a[OC_NC], b[OC_NC], c[OC_NC], inv[OC_NC];
            a[0] = l1;
            b[0] = l2;
#pragma unroll
            for (int k = 0; k < OC_NC; ++k) {
                c[k] = 0.5 * (a[k] + b[k]);
                inv[k] = 1.0 / c[k];
                if (2 * k + 2 < OC_NC) {
                    a[2 * k + 1] = a[k];
                    b[2 * k + 1] = c[k];
                    a[2 * k + 2] = c[k];
                    b[2 * k + 2] = b[k];
                }
            }
            double v[OC_NC], tot[OC_NC];
            // FP32 screen of the 15 volumes. Per element the FP32 term differs from
            // the FP64 one by at most 4.01 u hi <= 4.01 u (u = 2^-24: rounding of
            // ocP, 1/lmid, their product, and of hi; clamping is 1-Lipschitz),
            // plus 2e-15 for subnormal ocP while 1/lmid <= 1e30; a thread's FP32
            // sum of at most M terms adds (M - 1) u of its value. A decision on
            // the path the walk takes is certain when the screened volume is
            // farther than that bound from volfrac; otherwise the pass is redone
            // in FP64, so the lambda sequence is the FP64 bisection's.
            bool certain = true;
#pragma unroll
            for (int k = 0; k < OC_NC; ++k) certain = certain && c[k] >= 1e-30 && c[k] <= 1e30;
            if (certain) {
                float inv32[OC_NC], vf[OC_NC];
#pragma unroll
                for (int k = 0; k < OC_NC; ++k) {
                    inv32[k] = (float)inv[k];
                    vf[k] = 0.f;
                }
                for (long long i = i0; i < n; i += stride) {
                    if (passive && passive[i] != 0) continue;
                    const double xi = x[i];
                    const float o = (float)ocp[i], hi = (float)fmin(xi + move, 1.0), lo = (float)fmax(xi - move, 0.0);
#pragma unroll
                    for (int k = 0; k < OC_NC; ++k) vf[k] += fmaxf(fminf(o * inv32[k], hi), lo);
                }
#pragma unroll
                for (int k = 0; k < OC_NC; ++k) v[k] = (double)vf[k];
                if (!grid_totals<ONT, OC_NC>(v, partials, parity, bar, deadline, tot)) return;
                parity ^= 1;
                const double u = 0x1p-24, M = (double)((n + stride - 1) / stride);
                double a1 = l1, a2 = l2;
                int kk = 0, sk = steps;
                for (int lev = 0; lev < OC_DEPTH; ++lev) {
                    if (!((a2 - a1) / (a1 + a2) > tol && sk < maxit)) break;
                    const double bound = (double)nact * (4.01 * u + 2e-15) + 1.01 * (M - 1.0) * u * fabs(tot[kk]);
                    const double vol = (tot[kk] + pas_sum) / nd;
                    if (!(fabs(vol - volfrac) > 1.25 * bound / nd + 1e-13 * (fabs(vol) + volfrac))) {
                        certain = false;
                        break;
                    }
                    if (vol > volfrac) {
                        a1 = c[kk];
                        kk = 2 * kk + 2;
                    } else {
                        a2 = c[kk];
                        kk = 2 * kk + 1;
                    }
                    ++sk;
                }
            }
            if (!certain) {
#pragma unroll
                for (int k = 0; k < OC_NC; ++k) v[k] = 0.0;
                for (long long i = i0; i < n; i += stride) {
                    if (passive && passive[i] != 0) continue;
                    // max(max(min(min(t, x + m), 1), x - m), 0) = max(min(t, hi), lo) exactly
                    const double xi = x[i], o = ocp[i];
                    const double hi = fmin(xi + move, 1.0), lo = fmax(xi - move, 0.0);
#pragma unroll
                    for (int k = 0; k < OC_NC; ++k) v[k] += fmax(fmin(o * inv[k], hi), lo);
                }
                if (!grid_totals<ONT, OC_NC>(v, partials, parity, bar, deadline, tot)) return;
                parity ^= 1;
            }
            int k = 0;
            for (int lev = 0; lev < OC_DEPTH; ++lev) {
                if (!((l2 - l1) / (l1 + l2) > tol && steps < maxit)) break;
                lmid = c[k];
                if ((tot[k] + pas_sum) / nd > volfrac) {
                    l1 = lmid;
                    k = 2 * k + 2;
                } else {
                    l2 = lmid;
                    k = 2 * k + 1;
                }
                ++steps;
            }
        }
        if ((l2 - l1) / (l1 + l2) > tol) status = (int)TO_ENOTCONV;
        const double inv_lm = 1.0 / lmid;
        for (long long i = i0; i < n; i += stride) {
            if (passive && passive[i] != 0) continue;
            const double xi = x[i];
            x[i] = fmax(fmax(fmin(fmin(ocp[i] * inv_lm, xi + move), 1.0), xi - move), 0.0);
        }
    } else {
        lmid = 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        out->lm = lmid;
        out->steps = steps;
        out->status = status;
    }
}

// Explicit primal-dual OC (Appendix A): with the move/box limits lo, up and
// ocP as above, lm = sqrt(lambda) is iterated in closed form,
//   lm <- sum_M ocP / (n f - sum_U up - sum_L lo - passive volume),
// where U = {ocP / lm >= up}, L = {ocP / lm <= lo} \ U and M the rest (the
// primal map puts U at up, L at lo, M at ocP / lm), starting from lambda# and
// stopping when two iterates differ by at most tol (reading R21). Three grid
// sums per iteration; the final design is min(max(ocP / lm, lo), up).
__global__ void __launch_bounds__(ONT) k_oc_pd(long long n, double* __restrict__ x, const double* __restrict__ dc,
                                               const double* __restrict__ dV0, const int8_t* __restrict__ passive,
                                               long long nact, double move, double volfrac, double tol,
                                               int maxit, long long deadline, double* __restrict__ ocp,
                                               double* partials, GridBarrier* bar, OcOut* out) {
    const long long stride = (long long)gridDim.x * ONT;
    const long long i0 = (long long)blockIdx.x * ONT + threadIdx.x;
    int parity = 0;
    double s2[2] = {0.0, 0.0}, t2[2];
    for (long long i = i0; i < n; i += stride) {
        const bool act = !passive || passive[i] == 0;
        if (act) {
            const double o = x[i] * sqrt(fmax(0.0, -dc[i] / dV0[i]));
            ocp[i] = o;
            s2[0] += o;
        } else {
            s2[1] += x[i];
        }
    }
    if (!grid_totals<ONT, 2>(s2, partials, parity, bar, deadline, t2)) return;
    parity ^= 1;
    const double fixed_volume = t2[1];
    double lm = (t2[0] / (double)nact) / volfrac;
    int steps = 0, status = 0;
    if (lm > 0.0) {
        bool converged = false;
        while (steps < maxit) {
            double v[3] = {0.0, 0.0, 0.0}, tot[3];  // sum_U up, sum_L lo, sum_M ocP
            for (long long i = i0; i < n; i += stride) {
                if (passive && passive[i] != 0) continue;
                const double xi = x[i], o = ocp[i];
                const double up = fmin(xi + move, 1.0), lo = fmax(xi - move, 0.0);
                const double t = o / lm;
                if (t >= up)
                    v[0] += up;
                else if (t <= lo)
                    v[1] += lo;
                else
                    v[2] += o;
            }
            if (!grid_totals<ONT, 3>(v, partials, parity, bar, deadline, tot)) return;
            parity ^= 1;
            ++steps;
            const double num = tot[2], den = volfrac * (double)n - tot[0] - tot[1] - fixed_volume;
            if (!(num > 0.0 && den > 0.0)) break;
            const double lm_new = num / den;
            converged = fabs(lm_new - lm) <= tol;
            lm = lm_new;
            if (converged) break;
        }
        if (!converged) status = (int)TO_ENOTCONV;
        for (long long i = i0; i < n; i += stride) {
            if (passive && passive[i] != 0) continue;
            const double xi = x[i];
            x[i] = fmin(fmax(ocp[i] / lm, fmax(xi - move, 0.0)), fmin(xi + move, 1.0));
        }
    } else {
        lm = 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        out->lm = lm;
        out->steps = steps;
        out->status = status;
    }
}

// ----------------------------------------------- OC on the physical field --

__global__ void __launch_bounds__(256) k_ocf_prep(long long n, const double* __restrict__ x,
                                                  const double* __restrict__ dc, const double* __restrict__ dV0,
                                                  const int8_t* __restrict__ passive, long long nact, double volfrac,
                                                  double* __restrict__ ocp, OcfState* s, double* partials,
                                                  unsigned* counter) {
    double v[1] = {0.0}, tot[1];
    for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
        if (passive && passive[i] != 0) continue;
        const double o = x[i] * sqrt(fmax(0.0, -dc[i] / dV0[i]));
        ocp[i] = o;
        v[0] += o;
    }
    if (last_block_totals<256, 1>(v, partials, counter, tot) && threadIdx.x == 0) {
        const double l2 = (tot[0] / (double)nact) / volfrac;
        s->l1 = 0.0;
        s->l2 = l2;
        s->lmid = l2;
        s->phase = l2 > 0.0 ? 0 : 3;
        s->grows = s->steps = s->status = 0;
    }
}

// Candidate x(lm) of Eq. 14 at lm = l2 (growing) or the bracket midpoint.
__global__ void k_ocf_cand(long long n, const double* __restrict__ x, const double* __restrict__ ocp,
                           const int8_t* __restrict__ passive, double move, OcfState* s, double* __restrict__ xc) {
    const int phase = s->phase;
    if (phase >= 2) return;
    const double lm = phase == 0 ? s->l2 : 0.5 * (s->l1 + s->l2);
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) s->lmid = lm;
    if (i >= n) return;
    const double xi = x[i];
    xc[i] = (passive && passive[i] != 0) ? xi
                                         : fmax(fmax(fmin(fmin(ocp[i] / lm, xi + move), 1.0), xi - move), 0.0);
}

// Volume of the projected, filtered candidate; the last block moves the bracket.
__global__ void __launch_bounds__(256) k_ocf_vol(long long n, const double* __restrict__ xf, int ft, double eta0,
                                                 const double* eta_dev, double beta, double volfrac, double tol,
                                                 int maxit, OcfState* s, double* partials, unsigned* counter) {
    if (s->phase >= 2) return;  // uniform
    const double eta = eta_dev ? *eta_dev : eta0;
    const double tb = tanh(beta * eta), den = tb + tanh(beta * (1.0 - eta));
    double v[1] = {0.0}, tot[1];
    for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < n; i += (long long)gridDim.x * 256)
        v[0] += ft > 1 ? (tb + tanh(beta * (xf[i] - eta))) / den : xf[i];
    if (last_block_totals<256, 1>(v, partials, counter, tot) && threadIdx.x == 0) {
        const bool over = tot[0] / (double)n > volfrac;
        double l1 = s->l1, l2 = s->l2;
        if (s->phase == 0) {
            if (over && s->grows < 60) {
                l1 = l2;
                l2 = 2.0 * l2;
                s->grows += 1;
            } else {
                s->phase = 1;
            }
        } else {
            if (over)
                l1 = s->lmid;
            else
                l2 = s->lmid;
            s->steps += 1;
        }
        s->l1 = l1;
        s->l2 = l2;
        if (s->phase == 1 && !((l2 - l1) / (l1 + l2) > tol && s->steps < maxit)) {
            s->status = (l2 - l1) / (l1 + l2) > tol ? (int)TO_ENOTCONV : 0;
            s->phase = 2;
        }
    }
}

void launch_oc_filtered(const Dims& d, const FilterTaps& taps, char bc, const double* rHs, double rHs_const,
                        double* x, const double* dc, const double* dV0, const int8_t* passive, long long nact,
                        double move, double volfrac, int ft, double eta, const double* eta_dev, double beta,
                        double tol, int maxit, double* ocp, double* xc, double* xf, OcfState* sdev,
                        OcfState* shost, double* partials, unsigned* counter, OcOut* out, cudaStream_t st) {
    const long long n = d.nel;
    const int nbr = std::min(div_up(n, 256), 1024), nbe = div_up(n, 256);
    k_ocf_prep<<<nbr, 256, 0, st>>>(n, x, dc, dV0, passive, nact, volfrac, ocp, sdev, partials, counter);
    TOPO_CHECK_LAUNCH();
    const int cap = maxit + 64;  // growing (at most 60) and bisection steps
    for (int done = 0; done < cap;) {
        for (int k = 0; k < 4; ++k, ++done) {
            k_ocf_cand<<<nbe, 256, 0, st>>>(n, x, ocp, passive, move, sdev, xc);
            TOPO_CHECK_LAUNCH();
            launch_filter(d, taps, bc, rHs, rHs_const, xc, nullptr, xf, passive, xc, st);
            k_ocf_vol<<<nbr, 256, 0, st>>>(n, xf, ft, eta, eta_dev, beta, volfrac, tol, maxit, sdev, partials,
                                           counter);
            TOPO_CHECK_LAUNCH();
        }
        TOPO_CUDA(cudaMemcpyAsync(shost, sdev, sizeof(OcfState), cudaMemcpyDeviceToHost, st));
        TOPO_CUDA(cudaStreamSynchronize(st));
        if (shost->phase >= 2) break;
    }
    OcOut o{0.0, 0, 0};
    if (shost->phase == 2) {
        TOPO_CUDA(cudaMemcpyAsync(x, xc, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        o = OcOut{shost->lmid, shost->steps, shost->status};
    } else if (shost->phase < 2) {
        o.status = (int)TO_ENOTCONV;
    }
    TOPO_CUDA(cudaMemcpyAsync(out, &o, sizeof(OcOut), cudaMemcpyHostToDevice, st));
    TOPO_CUDA(cudaStreamSynchronize(st));
}

int oc_max_blocks() {
    int dev = 0, nsm = 0, per = 0;
    TOPO_CUDA(cudaGetDevice(&dev));
    TOPO_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    int per_pd = 0;
    TOPO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_oc, ONT, 0));
    TOPO_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_pd, k_oc_pd, ONT, 0));
    per = std::min(per, per_pd);
    return nsm * (per < 2 ? per : 2);
}

void launch_oc(long long n, double* x, const double* dc, const double* dV0, const int8_t* passive,
               long long nact, double move, double volfrac, double tol, int maxit, long long deadline,
               double* ocp, double* partials, GridBarrier* bar, OcOut* out, int nblocks,
               cudaStream_t st, int method) {
    TOPO_CUDA(cudaMemsetAsync(bar, 0, sizeof(GridBarrier), st));
    void* args[] = {&n, &x, &dc, &dV0, &passive, &nact, &move, &volfrac, &tol, &maxit, &deadline,
                    &ocp, &partials, &bar, &out};
    TOPO_CUDA(cudaLaunchCooperativeKernel((void*)(method == TO_OC_PRIMAL_DUAL ? k_oc_pd : k_oc), dim3(nblocks),
                                          dim3(ONT), args, 0, st));
    count_launches(1);
}

// ------------------------------------------------------- dots, fills --

constexpr int RNT = 256;

__global__ void __launch_bounds__(RNT) k_dot(long long n, const double* __restrict__ a,
                                             const double* __restrict__ b, double* out,
                                             double* partials, unsigned* counter) {
    double v[1] = {0.0}, tot[1];
    for (long long i = (long long)blockIdx.x * RNT + threadIdx.x; i < n; i += (long long)gridDim.x * RNT)
        v[0] += a[i] * (b ? b[i] : a[i]);
    if (last_block_totals<RNT, 1>(v, partials, counter, tot) && threadIdx.x == 0) out[0] = tot[0];
}

static int red_blocks(long long n) {
    int nb = div_up(n, RNT * 4);
    return nb < 1 ? 1 : (nb > 1024 ? 1024 : nb);
}

void launch_dot(long long n, const double* a, const double* b, double* out, double* partials,
                unsigned* counter, cudaStream_t st) {
    k_dot<<<red_blocks(n), RNT, 0, st>>>(n, a, b, out, partials, counter);
    TOPO_CHECK_LAUNCH();
}

__global__ void __launch_bounds__(RNT) k_change(long long n, const double* __restrict__ a, double* b,
                                                double* out, int copy, double* partials,
                                                unsigned* counter) {
    double v[2] = {0.0, 0.0}, tot[2];
    for (long long i = (long long)blockIdx.x * RNT + threadIdx.x; i < n; i += (long long)gridDim.x * RNT) {
        const double ai = a[i], di = ai - b[i];
        v[0] += di * di;
        v[1] += ai;
        if (copy) b[i] = ai;
    }
    if (last_block_totals<RNT, 2>(v, partials, counter, tot) && threadIdx.x == 0) {
        out[0] = tot[0];
        out[1] = tot[1];
    }
}

void launch_change(long long n, const double* a, double* b, double* out, int copy, double* partials,
                   unsigned* counter, cudaStream_t st) {
    k_change<<<red_blocks(n), RNT, 0, st>>>(n, a, b, out, copy, partials, counter);
    TOPO_CHECK_LAUNCH();
}

__global__ void k_fill(long long n, double* a, double v) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}
void launch_fill(long long n, double* a, double v, cudaStream_t st) {
    k_fill<<<div_up(n, 256), 256, 0, st>>>(n, a, v);
    TOPO_CHECK_LAUNCH();
}

__global__ void k_dv(long long n, const int8_t* passive, double v, double* dV) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dV[i] = (passive && passive[i] != 0) ? 0.0 : v;
}
void launch_dv(long long n, const int8_t* passive, double v, double* dV, cudaStream_t st) {
    k_dv<<<div_up(n, 256), 256, 0, st>>>(n, passive, v, dV);
    TOPO_CHECK_LAUNCH();
}

__global__ void k_mask_copy(long long n, const double* __restrict__ in, double* __restrict__ out,
                            const uint8_t* __restrict__ fixed) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = fixed[i] ? 0.0 : in[i];
}
void launch_mask_copy(long long n, const double* in, double* out, const uint8_t* fixed, cudaStream_t st) {
    k_mask_copy<<<div_up(n, 256), 256, 0, st>>>(n, in, out, fixed);
    TOPO_CHECK_LAUNCH();
}

// ----------------------------------------------------------------- PCG --

__global__ void __launch_bounds__(RNT) k_pcg_init(long long n, const double* __restrict__ b,
                                                  const double* __restrict__ Ax, double* __restrict__ x,
                                                  double* __restrict__ r, double* __restrict__ z,
                                                  double* __restrict__ p, const double* __restrict__ dinv,
                                                  const uint8_t* __restrict__ fixed, PcgScalars* s,
                                                  double* partials, unsigned* counter) {
    double v[3] = {0.0, 0.0, 0.0}, tot[3];
    for (long long i = (long long)blockIdx.x * RNT + threadIdx.x; i < n; i += (long long)gridDim.x * RNT) {
        const bool f = fixed[i] != 0;
        const double bi = f ? 0.0 : b[i];
        const double ri = f ? 0.0 : bi - Ax[i];
        if (f) x[i] = 0.0;
        const double zi = dinv[i] * ri;
        r[i] = ri;
        z[i] = zi;
        p[i] = zi;
        v[0] += ri * zi;
        v[1] += ri * ri;
        v[2] += bi * bi;
    }
    if (last_block_totals<RNT, 3>(v, partials, counter, tot) && threadIdx.x == 0) {
        s->rz = tot[0];
        s->rr = tot[1];
        s->bb = tot[2];
        s->iters = 0;
        s->done = (tot[1] <= s->rtol2 * tot[2]) ? 1 : 0;
        if (!isfinite(tot[1])) s->done = 3;
    }
}

void launch_pcg_init(long long n, const double* b, const double* Ax, double* x, double* r, double* z,
                     double* p, const double* dinv, const uint8_t* fixed, PcgScalars* s,
                     double* partials, unsigned* counter, cudaStream_t st) {
    k_pcg_init<<<red_blocks(n), RNT, 0, st>>>(n, b, Ax, x, r, z, p, dinv, fixed, s, partials, counter);
    TOPO_CHECK_LAUNCH();
}

__global__ void __launch_bounds__(RNT) k_pcg_update(long long n, double* __restrict__ x,
                                                    double* __restrict__ r, double* __restrict__ z,
                                                    const double* __restrict__ p,
                                                    const double* __restrict__ Ap,
                                                    const double* __restrict__ dinv, PcgScalars* s,
                                                    double* partials, unsigned* counter) {
    if (s->done) return;
    const double alpha = s->alpha;
    double v[2] = {0.0, 0.0}, tot[2];
    for (long long i = (long long)blockIdx.x * RNT + threadIdx.x; i < n; i += (long long)gridDim.x * RNT) {
        x[i] += alpha * p[i];
        const double ri = r[i] - alpha * Ap[i];
        r[i] = ri;
        const double zi = dinv[i] * ri;
        z[i] = zi;
        v[0] += ri * zi;
        v[1] += ri * ri;
    }
    if (last_block_totals<RNT, 2>(v, partials, counter, tot) && threadIdx.x == 0) {
        s->iters += 1;
        s->rr = tot[1];
        s->rz_new = tot[0];
        s->beta = tot[0] / s->rz;
        s->rz = tot[0];
        if (!isfinite(tot[1]))
            s->done = 3;
        else if (tot[1] <= s->rtol2 * s->bb)
            s->done = 1;
        else if (s->iters >= s->maxit)
            s->done = 2;
    }
}

void launch_pcg_update(long long n, double* x, double* r, double* z, const double* p, const double* Ap,
                       const double* dinv, PcgScalars* s, double* partials, unsigned* counter,
                       cudaStream_t st) {
    k_pcg_update<<<red_blocks(n), RNT, 0, st>>>(n, x, r, z, p, Ap, dinv, s, partials, counter);
    TOPO_CHECK_LAUNCH();
}

__global__ void k_pcg_dir(long long n, const double* __restrict__ z, double* __restrict__ p,
                          const PcgScalars* s) {
    if (s->done) return;
    const double beta = s->beta;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = z[i] + beta * p[i];
}

void launch_pcg_dir(long long n, const double* z, double* p, const PcgScalars* s, cudaStream_t st) {
    k_pcg_dir<<<div_up(n, 256), 256, 0, st>>>(n, z, p, s);
    TOPO_CHECK_LAUNCH();
}

}  // namespace topo
