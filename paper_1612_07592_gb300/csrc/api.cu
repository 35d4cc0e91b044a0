// api.cu -- the C ABI declared in include/pe.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <memory>
#include <mutex>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "physics.cuh"

using namespace pe;

struct pe_tables {
    HostTables host;
    TablesDev dev;
    void* dmem = nullptr;
    void* dmemq = nullptr;    // pair-row tables and guides of the FP32 emission branch
    int device = 0;
    // Bethe-Heitler tables, built and uploaded by the first call that needs them
    mutable std::mutex bh_mu;
    mutable std::vector<double> bh_sigma, bh_cdf;
    mutable double* bh_dev = nullptr;     // sigma_BH then the CDF, FP64
};

struct pe_run {
    RunDev dev;
    pe_run_params params;
    pe_buffers buf;
    const pe_tables* tables = nullptr;
    cudaStream_t stream = nullptr;
    int64_t steps_done = 0;
    void* jacc = nullptr;     // 1D PIC: the library's current sums of one step
    ~pe_run() {
        if (jacc) cudaFree(jacc);
    }
};

namespace {

thread_local std::string g_err;
std::atomic<int64_t> g_launches{0};

pe_status fail(pe_status s, const std::string& msg) {
    g_err = msg;
    return s;
}
pe_status cuda_fail(cudaError_t e, const char* where) {
    return fail(PE_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// largest value <= dt with 11 significant bits, so n * dt_hi is exact in float for n < 2^13
void split_dt(double dt, double* hi, double* lo) {
    int e;
    double m = std::frexp(dt, &e);
    double mh = std::floor(std::ldexp(m, 11));
    *hi = std::ldexp(mh, e - 11);
    *lo = dt - *hi;
}

}  // namespace

extern "C" const char* pe_last_error(void) { return g_err.c_str(); }
extern "C" int64_t pe_launch_count(void) { return g_launches.load(); }

extern "C" double pe_a0_from_intensity(double I_wcm2, double lambda_m, int polarisation) {
    double a = 0.855 * (lambda_m * 1e6) * std::sqrt(I_wcm2 / 1e18);
    return polarisation == PE_CP ? a / std::sqrt(2.0) : a;
}

struct pe_bw_tables {
    BwDev dev;
    void* dmem = nullptr;
    int device = 0;
};

extern "C" pe_status pe_bw_tables_create(int n_chi, double chi_min, double chi_max, int n_x, pe_bw_tables** out) {
    if (!out) return fail(PE_ERR_ARG, "pe_bw_tables_create: null out");
    *out = nullptr;
    if (n_chi < 2 || n_x < 2 || n_chi > 4096 || n_x > 4096 || !(chi_min > 0.0) || !(chi_max > chi_min) ||
        !std::isfinite(chi_max))
        return fail(PE_ERR_ARG, "pe_bw_tables_create: need 2 <= n_chi, n_x <= 4096 and 0 < chi_min < chi_max");
    std::vector<double> T(n_chi), cdf((size_t)n_chi * n_x);
    build_host_bw_tables(n_chi, chi_min, chi_max, n_x, T.data(), cdf.data());
    for (double v : T)
        if (!(v > 0.0) || !std::isfinite(v))
            return fail(PE_ERR_ARG, "pe_bw_tables_create: T(chi) underflows at chi_min; raise chi_min");
    // L_i = ln T_i + 8 / (3 chi_i), chi_i on the log grid (T is interpolated as exp(L - 8 / (3 chi)))
    std::vector<double> L(n_chi);
    std::vector<float> L32(n_chi);
    const double llo = std::log(chi_min), lhi = std::log(chi_max);
    for (int i = 0; i < n_chi; ++i) {
        const double ci = std::exp(llo + (lhi - llo) * (double)i / (double)(n_chi - 1));
        L[i] = std::log(T[i]) + 8.0 / (3.0 * ci);
        L32[i] = (float)L[i];
    }
    pe_bw_tables* t = new pe_bw_tables();
    cudaGetDevice(&t->device);
    const size_t b64 = sizeof(double) * ((size_t)n_chi + cdf.size()), b32 = sizeof(float) * (size_t)(n_chi + (n_chi & 1));
    cudaError_t e = cudaMalloc(&t->dmem, b64 + b32 + sizeof(unsigned long long));
    if (e != cudaSuccess) {
        delete t;
        return fail(PE_ERR_NOMEM, std::string("pe_bw_tables_create: cudaMalloc: ") + cudaGetErrorString(e));
    }
    double* dL = static_cast<double*>(t->dmem);
    double* dcdf = dL + n_chi;
    float* dL32 = reinterpret_cast<float*>(dcdf + cdf.size());
    e = cudaMemcpy(dL, L.data(), sizeof(double) * n_chi, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dcdf, cdf.data(), sizeof(double) * cdf.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dL32, L32.data(), sizeof(float) * n_chi, cudaMemcpyHostToDevice);
    unsigned long long* dbg = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(dL32) + b32);
    if (e == cudaSuccess) e = cudaMemset(dbg, 0, sizeof(unsigned long long));
    if (e != cudaSuccess) {
        cudaFree(t->dmem);
        delete t;
        return cuda_fail(e, "pe_bw_tables_create: upload");
    }
    BwDev& d = t->dev;
    d.L64 = dL; d.L32 = dL32; d.cdf64 = dcdf;
    d.dbg = dbg;
    d.T_last = T[n_chi - 1];
    d.chi_min = chi_min;
    d.ln_chi_min = llo;
    d.inv_dln_chi = (double)(n_chi - 1) / (lhi - llo);
    d.fT_last = (float)d.T_last; d.fchi_min = (float)chi_min; d.fln_chi_min = (float)llo;
    d.finv_dln_chi = (float)d.inv_dln_chi;
    d.f_last = (float)(n_chi - 1);
    d.n_chi = n_chi; d.n_x = n_x;
    *out = t;
    return PE_OK;
}

extern "C" pe_status pe_bw_tables_destroy(pe_bw_tables* t) {
    if (!t) return fail(PE_ERR_ARG, "pe_bw_tables_destroy: null");
    if (t->dmem) cudaFree(t->dmem);
    delete t;
    return PE_OK;
}

extern "C" pe_status pe_bw_tables_host(int n_chi, double chi_min, double chi_max, int n_x, double* T,
                                        double* cdf) {
    if (!T || !cdf) return fail(PE_ERR_ARG, "pe_bw_tables_host: null argument");
    if (n_chi < 2 || n_x < 2 || n_chi > 4096 || n_x > 4096 || !(chi_min > 0.0) || !(chi_max > chi_min) ||
        !std::isfinite(chi_max))
        return fail(PE_ERR_ARG, "pe_bw_tables_host: need 2 <= n_chi, n_x <= 4096 and 0 < chi_min < chi_max");
    build_host_bw_tables(n_chi, chi_min, chi_max, n_x, T, cdf);
    return PE_OK;
}

extern "C" pe_status pe_create_tables(const pe_table_params* p, pe_tables** out) {
    if (!p || !out) return fail(PE_ERR_ARG, "pe_create_tables: null argument");
    *out = nullptr;
    if (p->n_eta < 2 || p->n_y < 2 || p->n_E < 2 || p->n_s < 2 || p->n_eta > 4096 || p->n_y > 4096 ||
        p->n_E > 4096 || p->n_s > 4096)
        return fail(PE_ERR_ARG, "pe_create_tables: table sizes must be in [2, 4096]");
    if (!(p->eta_min > 0 && p->eta_max > p->eta_min && p->y_min > 0 && p->y_max > p->y_min &&
          p->gamma_min > 1 && p->gamma_max > p->gamma_min && p->photon_min_mc2 > 0))
        return fail(PE_ERR_ARG, "pe_create_tables: ranges must be positive and increasing (gamma_min > 1)");
    if (p->n_Z < 1 || p->n_Z > 16 || !p->Z) return fail(PE_ERR_ARG, "pe_create_tables: need 1..16 values of Z");
    for (int i = 0; i < p->n_Z; ++i)
        if (!(p->Z[i] >= 1.0 && p->Z[i] <= 120.0)) return fail(PE_ERR_ARG, "pe_create_tables: Z out of [1, 120]");

    pe_tables* t = new pe_tables();
    std::string err;
    if (!build_host_tables(*p, t->host, &err)) {
        delete t;
        return fail(PE_ERR_ARG, "pe_create_tables: " + err);
    }
    cudaGetDevice(&t->device);
    const HostTables& H = t->host;
    size_t n_h = H.h.size(), n_c = H.cdf.size(), n_sg = H.sigma.size(), n_b = H.bcdf.size();
    size_t n_all = n_h + n_c + n_sg + n_b;
    size_t bytes = n_all * (sizeof(double) + 2 * sizeof(float)) + 64;
    cudaError_t e = cudaMalloc(&t->dmem, bytes);
    if (e != cudaSuccess) {
        delete t;
        return fail(PE_ERR_NOMEM, std::string("pe_create_tables: cudaMalloc: ") + cudaGetErrorString(e));
    }
    std::vector<double> all64;
    all64.reserve(n_all);
    all64.insert(all64.end(), H.h.begin(), H.h.end());
    all64.insert(all64.end(), H.cdf.begin(), H.cdf.end());
    all64.insert(all64.end(), H.sigma.begin(), H.sigma.end());
    all64.insert(all64.end(), H.bcdf.begin(), H.bcdf.end());
    std::vector<float> all32(all64.begin(), all64.end());
    std::vector<float> all32lo(n_all);
    for (size_t k = 0; k < n_all; ++k) all32lo[k] = (float)(all64[k] - (double)all32[k]);
    double* d64 = static_cast<double*>(t->dmem);
    float* d32 = reinterpret_cast<float*>(d64 + n_all);
    float* d32lo = d32 + n_all;
    e = cudaMemcpy(d64, all64.data(), n_all * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d32, all32.data(), n_all * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d32lo, all32lo.data(), n_all * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(t->dmem);
        delete t;
        return cuda_fail(e, "pe_create_tables: cudaMemcpy");
    }
    TablesDev& D = t->dev;
    {
        // pair-row tables and guide tables (see internal.h)
        const int ne = p->n_eta, ny = p->n_y, nE = p->n_E, ns = p->n_s, nZ = p->n_Z;
        auto pow2 = [](int v) { int m = 1; while (m < v) m <<= 1; return m; };
        const int My = pow2(ny), Ms = pow2(ns);
        const size_t nq_n = (size_t)ne * ny, nq_b = (size_t)nZ * (nE - 1) * ns;
        const size_t ng_n = (size_t)ne * My, ng_b = (size_t)nZ * (nE - 1) * Ms;
        std::vector<float4> q((nq_n + nq_b));
        std::vector<short4> g(ng_n + ng_b);
        const float* c32 = all32.data() + n_h;
        const float* c32lo = all32lo.data() + n_h;
        const float* b32 = all32.data() + n_h + n_c + n_sg;
        const float* b32lo = all32lo.data() + n_h + n_c + n_sg;
        // out[m] = J(m / M) for m = 0..M, J(u) the largest j with hi[j] + lo[j] <= u (the
        // float pair summed exactly in double), -1 if none: column k counts from the first
        // m with m / M >= c_k (c_k M is exact, M a power of two), then a running maximum
        auto guide = [](const float* hi, const float* lo, int n, int M, short* out) {
            std::vector<int> mark(M + 1, -1);
            for (int k = 0; k < n; ++k) {
                double x = std::ceil(((double)hi[k] + (double)lo[k]) * M);
                if (x > M) continue;
                int m0 = x < 0 ? 0 : (int)x;
                mark[m0] = std::max(mark[m0], k);
            }
            int run = -1;
            for (int m = 0; m <= M; ++m) {
                run = std::max(run, mark[m]);
                out[m] = (short)run;
            }
        };
        auto fill = [&](float4* qd, short4* gd, const float* ah, const float* al, const float* bh, const float* bl,
                        int n, int M) {
            for (int j = 0; j < n; ++j) qd[j] = make_float4(ah[j], al[j], bh[j], bl[j]);
            std::vector<short> ja(M + 1), jb(M + 1);
            guide(ah, al, n, M, ja.data());
            guide(bh, bl, n, M, jb.data());
            for (int m = 0; m < M; ++m) gd[m] = make_short4(ja[m], jb[m], ja[m + 1], jb[m + 1]);
        };
        for (int i = 0; i < ne; ++i) {
            const size_t ra = (size_t)(i < ne - 1 ? i : ne) * ny, rb = (size_t)(i < ne - 1 ? i + 1 : ne) * ny;
            fill(q.data() + (size_t)i * ny, g.data() + (size_t)i * My, c32 + ra, c32lo + ra, c32 + rb, c32lo + rb,
                 ny, My);
        }
        for (int z = 0; z < nZ; ++z)
            for (int i = 0; i < nE - 1; ++i) {
                const size_t ra = ((size_t)z * nE + i) * ns, rb = ra + ns;
                const size_t pr = (size_t)z * (nE - 1) + i;
                fill(q.data() + nq_n + pr * ns, g.data() + ng_n + pr * Ms, b32 + ra, b32lo + ra, b32 + rb, b32lo + rb,
                     ns, Ms);
            }
        const size_t qbytes = q.size() * sizeof(float4), gbytes = g.size() * sizeof(short4);
        e = cudaMalloc(&t->dmemq, qbytes + gbytes);
        if (e == cudaSuccess) e = cudaMemcpy(t->dmemq, q.data(), qbytes, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(static_cast<char*>(t->dmemq) + qbytes, g.data(), gbytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(t->dmem);
            if (t->dmemq) cudaFree(t->dmemq);
            delete t;
            return cuda_fail(e, "pe_create_tables: guide tables");
        }
        const float4* dq = static_cast<const float4*>(t->dmemq);
        const short4* dg = reinterpret_cast<const short4*>(static_cast<const char*>(t->dmemq) + qbytes);
        D.cdfq = dq; D.bcdfq = dq + nq_n;
        D.gq = dg; D.bgq = dg + ng_n;
        D.M_y = My; D.M_s = Ms;
        D.fM_y = (float)My; D.fM_s = (float)Ms;
    }
    // the word after the three copies counts table indices found out of range (debug builds)
    D.dbg = reinterpret_cast<unsigned long long*>(d32lo + n_all);     // byte 16 n_all: 8-byte aligned
    e = cudaMemset(D.dbg, 0, sizeof(unsigned long long));
    if (e != cudaSuccess) {
        cudaFree(t->dmem);
        cudaFree(t->dmemq);
        delete t;
        return cuda_fail(e, "pe_create_tables: debug word");
    }
    D.h64 = d64; D.cdf64 = d64 + n_h; D.sig64 = D.cdf64 + n_c; D.bcdf64 = D.sig64 + n_sg;
    D.h32 = d32; D.cdf32 = d32 + n_h; D.sig32 = D.cdf32 + n_c; D.bcdf32 = D.sig32 + n_sg;
    D.cdf32lo = d32lo + n_h;
    D.bcdf32lo = d32lo + n_h + n_c + n_sg;
    D.n_eta = p->n_eta; D.n_y = p->n_y; D.n_E = p->n_E; D.n_s = p->n_s; D.n_Z = p->n_Z;
    TabC<double>& C = D.cd;
    C.eta_min = p->eta_min;
    C.ln_eta_min = std::log(p->eta_min);
    C.inv_dln_eta = (p->n_eta - 1) / (std::log(p->eta_max) - std::log(p->eta_min));
    C.ln_y_min = std::log(p->y_min);
    C.dln_y = (std::log(p->y_max) - std::log(p->y_min)) / (p->n_y - 1);
    C.y_min = p->y_min; C.y_max = p->y_max;
    C.ln_g_min = std::log(p->gamma_min);
    C.inv_dln_g = (p->n_E - 1) / (std::log(p->gamma_max) - std::log(p->gamma_min));
    C.photon_min = p->photon_min_mc2;
    C.h_classical = 5.0 * kPi / 3.0;
    C.eta_last = p->n_eta - 1;
    C.g_last = p->n_E - 1;
    C.s_step = 1.0 / (p->n_s - 1);
    C.ln_k_min = std::log(2.0);
    C.inv_dln_k = p->gamma_max > 2.0 ? (p->n_E - 1) / (std::log(p->gamma_max) - std::log(2.0)) : 0.0;
    const double* cs = &C.eta_min;
    float* cfp = &D.cf.eta_min;
    for (size_t k = 0; k < sizeof(TabC<double>) / sizeof(double); ++k) cfp[k] = (float)cs[k];
    *out = t;
    return PE_OK;
}

extern "C" pe_status pe_destroy_tables(pe_tables* t) {
    if (!t) return fail(PE_ERR_ARG, "pe_destroy_tables: null");
    if (t->dmem) cudaFree(t->dmem);
    if (t->dmemq) cudaFree(t->dmemq);
    if (t->bh_dev) cudaFree(t->bh_dev);
    delete t;
    return PE_OK;
}

namespace {
// the Bethe-Heitler tables of t on the host and, with upload, on t's device
pe_status ensure_bh(const pe_tables* t, bool upload) {
    std::lock_guard<std::mutex> lock(t->bh_mu);
    if (!(t->host.p.gamma_max > 2.0)) return fail(PE_ERR_ARG, "pair tables: gamma_max must exceed 2");
    if (t->bh_sigma.empty()) build_host_bh_tables(t->host, t->bh_sigma, t->bh_cdf);
    if (upload && !t->bh_dev) {
        const size_t n1 = t->bh_sigma.size(), n2 = t->bh_cdf.size();
        int cur = 0;
        cudaGetDevice(&cur);
        if (cur != t->device) cudaSetDevice(t->device);
        double* d = nullptr;
        cudaError_t e = cudaMalloc(&d, sizeof(double) * (n1 + n2));
        if (e == cudaSuccess) e = cudaMemcpy(d, t->bh_sigma.data(), sizeof(double) * n1, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d + n1, t->bh_cdf.data(), sizeof(double) * n2, cudaMemcpyHostToDevice);
        if (cur != t->device) cudaSetDevice(cur);
        if (e != cudaSuccess) {
            if (d) cudaFree(d);
            return cuda_fail(e, "pair tables: upload");
        }
        t->bh_dev = d;
    }
    return PE_OK;
}
}  // namespace

extern "C" pe_status pe_tables_export(const pe_tables* t, int which, int iz, double* out, int64_t cap,
                                      int64_t* n_out) {
    if (!t || !out) return fail(PE_ERR_ARG, "pe_tables_export: null argument");
    const HostTables& H = t->host;
    const pe_table_params& p = H.p;
    const double* src = nullptr;
    int64_t n = 0;
    if ((which >= 3 && which <= 6) && (iz < 0 || iz >= p.n_Z)) return fail(PE_ERR_ARG, "pe_tables_export: bad iz");
    if (which == 5 || which == 6) {
        pe_status st = ensure_bh(t, false);
        if (st != PE_OK) return st;
    }
    switch (which) {
        case 0: src = H.h.data(); n = p.n_eta; break;
        case 1: src = H.cdf.data(); n = (int64_t)p.n_eta * p.n_y; break;
        case 2: src = H.cdf.data() + (size_t)p.n_eta * p.n_y; n = p.n_y; break;
        case 3: src = H.sigma.data() + (size_t)iz * p.n_E; n = p.n_E; break;
        case 4: src = H.bcdf.data() + (size_t)iz * p.n_E * p.n_s; n = (int64_t)p.n_E * p.n_s; break;
        case 5: src = t->bh_sigma.data() + (size_t)iz * p.n_E; n = p.n_E; break;
        case 6: src = t->bh_cdf.data() + (size_t)iz * p.n_E * p.n_s; n = (int64_t)p.n_E * p.n_s; break;
        default: return fail(PE_ERR_ARG, "pe_tables_export: which must be 0..6");
    }
    if (n_out) *n_out = n;
    if (cap < n) return fail(PE_ERR_ARG, "pe_tables_export: output too small");
    std::memcpy(out, src, sizeof(double) * n);
    return PE_OK;
}

// The checks every entry point that takes a run description applies (`who` names the
// entry point in the message); *iz_out receives the index of the run's Z in the table set.
static pe_status check_run(const pe_tables* t, const pe_run_params* rp, int64_t n, const pe_buffers* b,
                           const char* who, int* iz_out) {
    const std::string w(who);
    if (!t || !rp || !b) return fail(PE_ERR_ARG, w + ": null argument");
    if (n < 0 || n >= (int64_t(1) << 31)) return fail(PE_ERR_ARG, w + ": n must be in [0, 2^31)");
    if ((int64_t)rp->id0 + n > (int64_t(1) << 32))
        return fail(PE_ERR_ARG, w + ": id0 + n must not exceed 2^32 (electron ids are 32-bit Philox counters)");
    if (rp->precision != PE_F32 && rp->precision != PE_F64) return fail(PE_ERR_ARG, w + ": precision");
    if (rp->geometry < PE_PLANE_1D || rp->geometry > PE_PIC_1D) return fail(PE_ERR_ARG, w + ": geometry");
    if (!(rp->lambda_m > 0 && rp->dt_over_T > 0 && rp->charge_state > 0 && rp->ne_over_nc >= 0 &&
          rp->ramp_periods > 0 && rp->flat_s >= 0))
        return fail(PE_ERR_ARG, w + ": lambda, dt, charge state, ramp must be positive; n_e, flat top >= 0");
    if (rp->geometry == PE_PIC_1D) {
        if (rp->n_cells < 4 || rp->n_cells > PE_PIC_MAX_CELLS)
            return fail(PE_ERR_ARG, w + ": n_cells must be in [4, PE_PIC_MAX_CELLS = 4096]");
        if (n > 0 && (!b->grid || !aligned16(b->grid))) return fail(PE_ERR_ARG, w + ": PIC grid buffer");
        const double L_m = rp->n_cells * rp->dt_over_T * rp->lambda_m;       // n_cells dx, dx = c dt
        if (!(rp->slab_x0_m > 0 && rp->slab_x0_m + rp->slab_thick_m < L_m))
            return fail(PE_ERR_ARG, w + ": the slab must lie inside the PIC grid (0, n_cells c dt)");
    }
    if (rp->polarisation != PE_LP_Y && rp->polarisation != PE_CP) return fail(PE_ERR_ARG, w + ": polarisation");
    if (rp->init_dist < PE_REST || rp->init_dist > PE_CALLER) return fail(PE_ERR_ARG, w + ": init_dist");
    if (rp->geometry == PE_GAUSS_2D && !(rp->w0_m > 0)) return fail(PE_ERR_ARG, w + ": w0");
    if (rp->init_dist == PE_MAXWELL_JUTTNER && !(rp->T_mev > 0)) return fail(PE_ERR_ARG, w + ": T_mev");
    if (rp->init_dist == PE_BEAM && !(rp->beam_gamma >= 1)) return fail(PE_ERR_ARG, w + ": beam_gamma");
    if (!(rp->reflect_r >= 0 && rp->reflect_r <= 1)) return fail(PE_ERR_ARG, w + ": reflect_r must be in [0, 1]");
    if (rp->reflect_r > 0 && rp->geometry != PE_PLANE_1D)
        return fail(PE_ERR_ARG, w + ": a reflected wave needs geometry PE_PLANE_1D");
    if (rp->brems_method != PE_BREMS_DIRECT && rp->brems_method != PE_BREMS_NULL)
        return fail(PE_ERR_ARG, w + ": brems_method");
    if (rp->brems_method == PE_BREMS_NULL && n > 0 && (!b->brems_wait || !aligned16(b->brems_wait)))
        return fail(PE_ERR_ARG, w + ": PE_BREMS_NULL needs a 16-byte aligned brems_wait buffer");
    if (n > 0) {
        if (!b->x || !b->y || !b->ux || !b->uy || !b->uz || !b->tau || !b->hist || !b->tally)
            return fail(PE_ERR_ARG, w + ": null buffer");
        const void* ps[] = {b->x, b->y, b->ux, b->uy, b->uz, b->tau, b->hist, b->tally};
        for (const void* q : ps)
            if (!aligned16(q)) return fail(PE_ERR_ARG, w + ": buffers must be 16-byte aligned");
    }
    if (!b->hist || !b->tally) return fail(PE_ERR_ARG, w + ": null hist/tally");
    if (b->events && !aligned16(b->events)) return fail(PE_ERR_ARG, w + ": events misaligned");
    if (b->photon_capacity < 0 || (b->photon_capacity > 0 && (!b->photons || !aligned16(b->photons))))
        return fail(PE_ERR_ARG, w + ": photon buffer");
    int iz = -1;
    for (int k = 0; k < t->host.p.n_Z; ++k)
        if (std::fabs(t->host.Z[k] - rp->Z) < 1e-9) iz = k;
    if (iz < 0) return fail(PE_ERR_ARG, w + ": Z is not in the table set");
    *iz_out = iz;
    return PE_OK;
}

// The device description of a checked run: buffers, the per-step constants of its
// laser, target and step in normalised units, the null-collision majorant and, for
// PE_PIC_1D, the grid and the macro-electron weight.  The step index (step0) is 0 and
// the PIC current sums (jacc) are unset: the caller supplies both.
static void describe_run(const pe_tables* t, const pe_run_params* rp, int64_t n, const pe_buffers* b, int iz,
                         RunDev& d) {
    std::memset(&d, 0, sizeof(d));
    d.x = b->x; d.y = b->y; d.ux = b->ux; d.uy = b->uy; d.uz = b->uz;
    d.tau = b->tau;
    d.photons = static_cast<uint8_t*>(b->photons);
    d.hist = static_cast<unsigned long long*>(b->hist);
    d.tally = static_cast<unsigned long long*>(b->tally);
    d.events = static_cast<unsigned long long*>(b->events);
    d.n = n;
    d.capacity = b->photon_capacity;
    d.step0 = 0;
    StepC<double>& c = d.c;
    const double kl = 2.0 * kPi / rp->lambda_m;
    c.dt = rp->dt_over_T * 2.0 * kPi;
    split_dt(c.dt, &c.dt_hi, &c.dt_lo);
    const double E_S = kMec2MeV * rp->lambda_m / (2.0 * kPi * kHbarcMeVm);
    c.inv_ES = 1.0 / E_S;
    c.ncs_coef = std::sqrt(3.0) * kAlpha / (2.0 * kPi) * E_S * c.dt;
    c.bw_coef = kAlpha * E_S * c.dt;
    const double n_c = kPi / (kRe * rp->lambda_m * rp->lambda_m);
    const double n_i = rp->ne_over_nc * n_c / rp->charge_state;
    c.K_br = n_i * kAlpha * kRe * kRe * (c.dt / kl);
    c.x0 = rp->slab_x0_m * kl;
    c.x1 = (rp->slab_x0_m + rp->slab_thick_m) * kl;
    c.yh = rp->y_half_m * kl;
    c.box0 = rp->box_x_m[0] * kl;
    c.box1 = rp->box_x_m[1] * kl;
    c.inv_log_emax = 1.0 / std::log(kHistEmaxMeV / kMec2MeV);
    c.a0 = rp->a0;
    c.w0 = rp->w0_m * kl;
    c.zr = 0.5 * c.w0 * c.w0;
    c.inv_zr = c.zr > 0 ? 1.0 / c.zr : 0.0;
    c.inv_w0sq = c.w0 > 0 ? 1.0 / (c.w0 * c.w0) : 0.0;
    c.xf = rp->focus_x_m * kl;
    c.phi_r = 2.0 * kPi * rp->ramp_periods;
    c.phi_f = 2.0 * kPi * rp->flat_s * kC / rp->lambda_m;
    c.k_env = 0.5 * kPi / c.phi_r;
    for (int k = 0; k < 3; ++k) { c.E_const[k] = rp->E_const[k]; c.B_const[k] = rp->B_const[k]; }
    c.refl_r = rp->reflect_r;
    const double xm2 = 2.0 * rp->mirror_x_m * kl;
    // 2 x_m = hi + lo with hi on dt_hi's grid (multiples of its last bit), so that the FP32 phase
    // of the reflected pulse forms n dt_hi - hi exactly (both on that grid, fewer than 2^24
    // steps of it); a mirror beyond that range takes the nearest float.  hi + lo is 2 x_m exactly.
    {
        int e;
        std::frexp(c.dt, &e);
        const double q = std::ldexp(1.0, e - 11);
        c.xm2_hi = std::nearbyint(xm2 / q) * q;
        if (!(std::fabs(c.xm2_hi) < std::ldexp(q, 23))) c.xm2_hi = (double)(float)xm2;
        c.xm2_lo = xm2 - c.xm2_hi;
    }
    // null collisions: majorant from the largest tabulated sigma_Z (beta <= 1)
    double smax = 0;
    for (int i = 0; i < t->host.p.n_E; ++i) smax = std::max(smax, t->host.sigma[(size_t)iz * t->host.p.n_E + i]);
    d.x_hat = c.K_br * smax;
    c.P_hat = -std::expm1(-d.x_hat);
    d.brems_method = rp->brems_method;
    d.wait = rp->brems_method == PE_BREMS_NULL ? static_cast<uint32_t*>(b->brems_wait) : nullptr;
    d.fk = field_kind(rp->geometry, rp->polarisation, rp->reflect_r > 0);
    d.geometry = rp->geometry;
    d.polarisation = rp->polarisation;
    d.enable_ncs = rp->enable_ncs;
    d.enable_brems = rp->enable_brems;
    d.box_enable = rp->box_enable;
    if (rp->geometry == PE_PIC_1D) {
        // electrons leaving the grid are removed by the PIC kernel after depositing their
        // last move; each carries the areal density n_e d / n
        d.box_enable = 0;
        c.box0 = 0.0;
        c.box1 = rp->n_cells * c.dt;
        const double w = n > 0 ? rp->ne_over_nc * rp->slab_thick_m * kl / (double)n : 0.0;
        c.pic_kx = w / c.dt / 68719476736.0;
        c.pic_kyz = -w / c.dt / 68719476736.0;
        d.grid = b->grid;
        d.n_cells = rp->n_cells;
    }
    d.iz = iz;
    d.run_id = rp->run_id;
    d.id0 = rp->id0;
    d.seed_lo = (uint32_t)(rp->seed & 0xffffffffu);
    d.seed_hi = (uint32_t)(rp->seed >> 32);
}

// A run on the caller's buffers.  resume = false: a new run (initial state drawn unless
// PE_CALLER, histograms, tallies and events cleared, PIC grid set up).  resume = true: the
// buffers already hold the state of step `step0` (a checkpoint) and are taken as they are.
static pe_status make_run(const pe_tables* t, const pe_run_params* rp, int64_t n, const pe_buffers* b, void* stream,
                          bool resume, int64_t step0, pe_run** out) {
    if (!out) return fail(PE_ERR_ARG, "pe_init_particles: null argument");
    *out = nullptr;
    if (step0 < 0 || step0 >= (int64_t(1) << 32)) return fail(PE_ERR_ARG, "pe_resume_particles: step0 out of range");
    int iz = -1;
    pe_status st = check_run(t, rp, n, b, resume ? "pe_resume_particles" : "pe_init_particles", &iz);
    if (st != PE_OK) return st;

    pe_run* r = new pe_run();
    r->params = *rp;
    r->buf = *b;
    r->tables = t;
    r->stream = static_cast<cudaStream_t>(stream);
    RunDev& d = r->dev;
    describe_run(t, rp, n, b, iz, d);

    r->steps_done = step0;
    cudaError_t e = cudaSuccess;
    if (!resume) {
        e = cudaMemsetAsync(b->hist, 0, sizeof(uint64_t) * PE_HIST_WORDS, r->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->tally, 0, sizeof(uint64_t) * PE_TALLY_WORDS, r->stream);
        if (e == cudaSuccess && b->events && n > 0) e = cudaMemsetAsync(b->events, 0, sizeof(uint64_t) * n, r->stream);
    }
    if (e != cudaSuccess) {
        delete r;
        return cuda_fail(e, "pe_init_particles: cudaMemsetAsync");
    }
    double theta = rp->T_mev / kMec2MeV;
    double beam_u = rp->init_dist == PE_BEAM ? std::sqrt(rp->beam_gamma * rp->beam_gamma - 1.0) : 0.0;
    if (n > 0 && !resume) {
        launch_init(d, rp->precision, rp->init_dist, theta, beam_u, r->stream);
        g_launches++;
        e = cudaGetLastError();
        if (e != cudaSuccess) {
            delete r;
            return cuda_fail(e, "pe_init_particles: k_init");
        }
    }
    if (rp->geometry == PE_PIC_1D && n > 0) {
        // zero fields, the ion charge of the neutral start, cleared current sums
        const size_t rs = rp->precision == PE_F32 ? 4 : 8;
        // 3 n_cells current sums and one word that counts the CTAs done with a step
        e = cudaMalloc(&r->jacc, sizeof(unsigned long long) * (3 * (size_t)rp->n_cells + 1));
        if (e != cudaSuccess) {
            r->jacc = nullptr;
            delete r;
            return fail(PE_ERR_NOMEM, std::string("pe_init_particles: PIC current sums: ") + cudaGetErrorString(e));
        }
        d.jacc = static_cast<unsigned long long*>(r->jacc);
        e = cudaMemsetAsync(r->jacc, 0, sizeof(unsigned long long) * (3 * (size_t)rp->n_cells + 1), r->stream);
        if (e == cudaSuccess && !resume)
            e = cudaMemsetAsync(b->grid, 0, rs * (size_t)PE_PIC_GRID_WORDS(rp->n_cells), r->stream);
        if (e == cudaSuccess && !resume) {
            launch_pic_rho(d, rp->precision, r->stream);
            g_launches += 2;
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) {
            delete r;
            return cuda_fail(e, "pe_init_particles: PIC grid");
        }
    }
    *out = r;
    return PE_OK;
}

extern "C" pe_status pe_init_particles(const pe_tables* t, const pe_run_params* rp, int64_t n,
                                       const pe_buffers* b, void* stream, pe_run** out) {
    return make_run(t, rp, n, b, stream, false, 0, out);
}

extern "C" pe_status pe_resume_particles(const pe_tables* t, const pe_run_params* rp, int64_t n,
                                         const pe_buffers* b, int64_t step0, void* stream, pe_run** out) {
    return make_run(t, rp, n, b, stream, true, step0, out);
}

// One persistent launch of a step call: the runs of one field kind, one chunk of
// at most steps_per_launch steps starting `offset` steps into the call.
struct PlanLaunch {
    int prec = PE_F32, grid = 0, block = 0, smem = 0, steps = 0;
    int64_t offset = 0;
    std::vector<int> idx;                       // positions in the runs array
    std::unique_ptr<BatchDevT<float>> bf;
    std::unique_ptr<BatchDevT<double>> bd;
};
struct Plan {
    std::vector<PlanLaunch> launches;
};

static void set_step0(PlanLaunch& L, pe_run* const* runs, int64_t base_extra) {
    for (size_t k = 0; k < L.idx.size(); ++k) {
        int64_t s0 = runs[L.idx[k]]->steps_done + base_extra + L.offset;
        if (L.prec == PE_F32) L.bf->runs[k].step0 = s0; else L.bd->runs[k].step0 = s0;
    }
}

// persistent launches (grouped by field kind, chunked by steps_per_launch)
static pe_status build_plan(pe_run* const* runs, int n_runs, int64_t n_steps, const pe_launch_config* cfg,
                            Plan& plan) {
    const pe_tables* t = runs[0]->tables;
    int prec = runs[0]->params.precision;
    int block = (cfg && cfg->block > 0) ? cfg->block : 256;
    if (block % 64 || block > 256) return fail(PE_ERR_ARG, "pe_step: block must be 64, 128, 192 or 256");
    int K = (cfg && cfg->steps_per_launch > 0) ? cfg->steps_per_launch : (int)std::min<int64_t>(n_steps, 4096);
    if (K < 1) K = 1;
    int dev;
    cudaGetDevice(&dev);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int smem = persistent_smem_bytes(t->dev, prec);
    if (smem > 200 * 1024)
        return fail(PE_ERR_ARG, "pe_step: rate tables (n_eta + n_Z * n_E) too large for shared memory");
    for (int fk = 0; fk < kFieldKinds; ++fk) {
        std::vector<int> idx;
        for (int k = 0; k < n_runs; ++k)
            if (runs[k]->dev.fk == fk) idx.push_back(k);
        if (idx.empty()) continue;
        int m = (int)idx.size();
        int64_t tile_start[PE_MAX_BATCH + 1];
        tile_start[0] = 0;
        for (int k = 0; k < m; ++k) tile_start[k + 1] = tile_start[k] + (runs[idx[k]]->dev.n + block - 1) / block;
        int64_t n_tiles = tile_start[m];
        if (n_tiles == 0) continue;
        // default grid: three resident waves of the paired kernel (plane wave, 2D focus), twice the
        // resident CTAs of the one-electron kernel, so the block scheduler evens out tiles of unequal cost
        int per_sm = (cfg && cfg->ctas_per_sm > 0) ? cfg->ctas_per_sm
                                                  : (prec == PE_F32 ? default_ctas_per_sm_f32(fk, block, smem, K)
                                                                    : 2 * persistent_occupancy_f64(block, smem));
        if (per_sm < 1) per_sm = 1;
        int grid = (int)std::min<int64_t>(n_tiles, (int64_t)sms * per_sm);
        for (int64_t done = 0; done < n_steps; done += K) {
            PlanLaunch L;
            L.prec = prec;
            L.grid = grid;
            L.block = block;
            L.smem = smem;
            L.steps = (int)std::min<int64_t>(K, n_steps - done);
            L.offset = done;
            L.idx = idx;
            if (prec == PE_F32) {
                L.bf.reset(new BatchDevT<float>());
                std::memset(L.bf.get(), 0, sizeof(BatchDevT<float>));
                L.bf->n_runs = m;
                L.bf->tile = block;
                for (int k = 0; k <= m; ++k) L.bf->tile_start[k] = tile_start[k];
                for (int k = 0; k < m; ++k) L.bf->runs[k] = to_float(runs[idx[k]]->dev);
            } else {
                L.bd.reset(new BatchDevT<double>());
                std::memset(L.bd.get(), 0, sizeof(BatchDevT<double>));
                L.bd->n_runs = m;
                L.bd->tile = block;
                for (int k = 0; k <= m; ++k) L.bd->tile_start[k] = tile_start[k];
                for (int k = 0; k < m; ++k) L.bd->runs[k] = runs[idx[k]]->dev;
            }
            plan.launches.push_back(std::move(L));
        }
    }
    return PE_OK;
}

static pe_status check_batch(pe_run* const* runs, int n_runs, int64_t n_steps) {
    if (!runs || n_runs < 1 || n_runs > PE_MAX_BATCH) return fail(PE_ERR_ARG, "pe_step: need 1..64 runs");
    if (n_steps < 0) return fail(PE_ERR_ARG, "pe_step: n_steps < 0");
    for (int k = 0; k < n_runs; ++k)
        if (!runs[k]) return fail(PE_ERR_ARG, "pe_step: null run");
    for (int k = 1; k < n_runs; ++k) {
        if (runs[k]->tables != runs[0]->tables)
            return fail(PE_ERR_STATE, "pe_step: runs of a batch must share one table set");
        if (runs[k]->params.precision != runs[0]->params.precision)
            return fail(PE_ERR_STATE, "pe_step: runs of a batch must share precision");
    }
    for (int k = 0; k < n_runs; ++k)
        if (runs[k]->steps_done + n_steps >= (int64_t(1) << 32))
            return fail(PE_ERR_ARG, "pe_step: step index would exceed 2^32");
    if (n_runs > 1)
        for (int k = 0; k < n_runs; ++k)
            if (runs[k]->dev.fk == FK_PIC) return fail(PE_ERR_STATE, "pe_step: a PE_PIC_1D run steps alone");
    return PE_OK;
}

extern "C" pe_status pe_step_ex(pe_run* const* runs, int n_runs, int64_t n_steps, const pe_launch_config* cfg) {
    pe_status st0 = check_batch(runs, n_runs, n_steps);
    if (st0 != PE_OK) return st0;
    const pe_tables* t = runs[0]->tables;
    int prec = runs[0]->params.precision;
    if (n_steps == 0) return PE_OK;
    cudaStream_t s = runs[0]->stream;

    if (runs[0]->dev.fk == FK_PIC) {
        // the grid changes every step: a particle launch and a field launch per step
        pe_run* r = runs[0];
        int dev, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        RunDev d = r->dev;
        if (d.n > 0) {
            for (int64_t k = 0; k < n_steps; ++k) {
                d.step0 = r->steps_done + k;
                launch_pic_step(t->dev, d, prec, sms, s);
                g_launches += 1;
            }
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "pe_step: PIC step");
        r->steps_done += n_steps;
        return PE_OK;
    }
    if (n_runs == 1 && prec == PE_F64 && !(cfg && cfg->steps_per_launch > 0)) {
        pe_run* r = runs[0];
        RunDev d = r->dev;
        for (int64_t k = 0; k < n_steps; ++k) {
            d.step0 = r->steps_done + k;
            launch_step_plain_f64(t->dev, d, s);
            g_launches++;
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "pe_step: k_step_plain");
        r->steps_done += n_steps;
        return PE_OK;
    }

    Plan plan;
    pe_status st = build_plan(runs, n_runs, n_steps, cfg, plan);
    (void)prec;
    if (st != PE_OK) return st;
    for (PlanLaunch& L : plan.launches) {
        set_step0(L, runs, 0);
        if (L.prec == PE_F32)
            launch_step_persistent_f32(t->dev, *L.bf, L.steps, L.grid, L.block, s);
        else
            launch_step_persistent_f64(t->dev, *L.bd, L.steps, L.grid, L.block, s);
        g_launches++;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "pe_step: k_step_persistent");
    for (int k = 0; k < n_runs; ++k) runs[k]->steps_done += n_steps;
    return PE_OK;
}

extern "C" pe_status pe_step(pe_run* const* runs, int n_runs, int64_t n_steps) {
    return pe_step_ex(runs, n_runs, n_steps, nullptr);
}

static double fx_value(const uint64_t* w, int i) {
    return (double)w[i + 1] + (double)w[i] * 0x1.0p-64;
}

extern "C" pe_status pe_tally(pe_run* r, pe_tally_out* out) {
    if (!r || !out) return fail(PE_ERR_ARG, "pe_tally: null argument");
    cudaError_t e = cudaStreamSynchronize(r->stream);
    if (e != cudaSuccess) return cuda_fail(e, "pe_tally: stream");
    e = cudaMemcpy(out->tally, r->buf.tally, sizeof(out->tally), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(out->hist, r->buf.hist, sizeof(out->hist), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "pe_tally: copy");
    out->n_particles = r->dev.n;
    out->steps_done = r->steps_done;
    uint64_t np = out->tally[PE_T_N_PHOTONS];
    out->photons_stored = (int64_t)std::min<uint64_t>(np, (uint64_t)r->buf.photon_capacity);
    double killed = (double)out->tally[PE_T_N_KILLED];
    out->live_particle_steps = ((double)r->dev.n - killed) * (double)r->steps_done + (double)out->tally[PE_T_KILLED_STEPS];
    out->e_ncs_stored = fx_value(out->tally, PE_T_E_NCS_STORED);
    out->e_ncs_below = fx_value(out->tally, PE_T_E_NCS_BELOW);
    out->e_br_stored = fx_value(out->tally, PE_T_E_BR_STORED);
    out->e_br_below = fx_value(out->tally, PE_T_E_BR_BELOW);
    out->e_recoil_ncs = fx_value(out->tally, PE_T_E_RECOIL_NCS);
    out->e_recoil_br = fx_value(out->tally, PE_T_E_RECOIL_BR);
    if (out->tally[PE_T_N_WAIT_TIMEOUT])
        return fail(PE_ERR_TIMEOUT, "pe_tally: a device wait for staged particle state ran out");
    if (np > (uint64_t)r->buf.photon_capacity)
        return fail(PE_ERR_BUFFER_FULL, "pe_tally: photon buffer overflowed (counts are exact)");
    return PE_OK;
}

extern "C" pe_status pe_electron_spectrum(pe_run* r, int n_bins, double e_min_mev, double e_max_mev, void* counts) {
    if (!r || !counts) return fail(PE_ERR_ARG, "pe_electron_spectrum: null argument");
    if (n_bins < 1 || n_bins > 4096) return fail(PE_ERR_ARG, "pe_electron_spectrum: n_bins must be in [1, 4096]");
    if (!(e_min_mev > 0 && e_max_mev > e_min_mev)) return fail(PE_ERR_ARG, "pe_electron_spectrum: energy range");
    if (!aligned16(counts)) return fail(PE_ERR_ARG, "pe_electron_spectrum: counts must be 16-byte aligned");
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * (size_t)n_bins, r->stream);
    if (e != cudaSuccess) return cuda_fail(e, "pe_electron_spectrum");
    launch_electron_spectrum(r->dev, r->params.precision, e_min_mev, e_max_mev, n_bins,
                             static_cast<unsigned long long*>(counts), r->stream);
    g_launches++;
    e = cudaGetLastError();
    return e == cudaSuccess ? PE_OK : cuda_fail(e, "pe_electron_spectrum");
}

extern "C" pe_status pe_photon_map(pe_run* r, int nx, double x_min_m, double x_max_m, int ne, double e_min_mev,
                                   double e_max_mev, void* counts) {
    if (!r || !counts) return fail(PE_ERR_ARG, "pe_photon_map: null argument");
    if (nx < 1 || ne < 1 || (int64_t)nx * ne > (int64_t(1) << 24))
        return fail(PE_ERR_ARG, "pe_photon_map: nx, ne >= 1 and nx * ne <= 2^24");
    if (!(x_max_m > x_min_m && e_min_mev > 0 && e_max_mev > e_min_mev))
        return fail(PE_ERR_ARG, "pe_photon_map: ranges");
    if (!aligned16(counts)) return fail(PE_ERR_ARG, "pe_photon_map: counts must be 16-byte aligned");
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * (size_t)nx * ne, r->stream);
    if (e != cudaSuccess) return cuda_fail(e, "pe_photon_map");
    const double kl = 2.0 * kPi / r->params.lambda_m;
    launch_photon_map(r->dev, x_min_m * kl, x_max_m * kl, nx, e_min_mev, e_max_mev, ne,
                      static_cast<unsigned long long*>(counts), r->stream);
    g_launches++;
    e = cudaGetLastError();
    return e == cudaSuccess ? PE_OK : cuda_fail(e, "pe_photon_map");
}

extern "C" pe_status pe_pair_transport(pe_run* r, const void* photons, int64_t n_photons, int64_t step_end,
                                        void* pairs, int64_t capacity, void* tally, int method) {
    if (!r || !tally || (n_photons > 0 && !photons) || (capacity > 0 && !pairs))
        return fail(PE_ERR_ARG, "pe_pair_transport: null argument");
    if (method != PE_PAIR_DIRECT && method != PE_PAIR_FREE_PATH)
        return fail(PE_ERR_ARG, "pe_pair_transport: method must be PE_PAIR_DIRECT or PE_PAIR_FREE_PATH");
    if (n_photons < 0 || n_photons >= (int64_t(1) << 31) || capacity < 0)
        return fail(PE_ERR_ARG, "pe_pair_transport: n_photons must be in [0, 2^31), capacity >= 0");
    if ((reinterpret_cast<uintptr_t>(photons) & 3u) || (reinterpret_cast<uintptr_t>(pairs) & 3u) ||
        (reinterpret_cast<uintptr_t>(tally) & 7u))
        return fail(PE_ERR_ARG, "pe_pair_transport: misaligned buffer");
    if (step_end < 0) step_end = r->steps_done;
    if (step_end > r->steps_done) return fail(PE_ERR_ARG, "pe_pair_transport: step_end beyond the run's steps");
    pe_status st = ensure_bh(r->tables, true);
    if (st != PE_OK) return st;
    cudaError_t e = cudaMemsetAsync(tally, 0, sizeof(unsigned long long) * PE_PAIR_TALLY_WORDS, r->stream);
    if (e != cudaSuccess) return cuda_fail(e, "pe_pair_transport");
    if (n_photons == 0) return PE_OK;
    TablesDev D = r->tables->dev;
    D.bhsig64 = r->tables->bh_dev;
    D.bhcdf64 = r->tables->bh_dev + r->tables->bh_sigma.size();
    launch_pair_transport(D, r->dev, photons, n_photons, step_end, pairs, capacity,
                          static_cast<unsigned long long*>(tally), method, r->stream);
    g_launches++;
    e = cudaGetLastError();
    return e == cudaSuccess ? PE_OK : cuda_fail(e, "pe_pair_transport");
}

extern "C" pe_status pe_bw_transport(pe_run* r, const pe_bw_tables* bw, const void* photons, int64_t n_photons,
                                      int64_t step_end, void* pairs, int64_t capacity, void* tally) {
    if (!r || !bw || !tally || (n_photons > 0 && !photons) || (capacity > 0 && !pairs))
        return fail(PE_ERR_ARG, "pe_bw_transport: null argument");
    if (r->dev.fk == FK_PIC)
        return fail(PE_ERR_STATE, "pe_bw_transport: a PE_PIC_1D run's self-consistent fields are not stored");
    if (n_photons < 0 || n_photons >= (int64_t(1) << 31) || capacity < 0)
        return fail(PE_ERR_ARG, "pe_bw_transport: n_photons must be in [0, 2^31), capacity >= 0");
    if ((reinterpret_cast<uintptr_t>(photons) & 3u) || (reinterpret_cast<uintptr_t>(pairs) & 3u) ||
        (reinterpret_cast<uintptr_t>(tally) & 7u))
        return fail(PE_ERR_ARG, "pe_bw_transport: misaligned buffer");
    if (step_end < 0) step_end = r->steps_done;
    if (step_end > r->steps_done) return fail(PE_ERR_ARG, "pe_bw_transport: step_end beyond the run's steps");
    if (r->params.precision == PE_F32 && step_end > 8192)
        return fail(PE_ERR_ARG, "pe_bw_transport: FP32 runs follow photons for at most 8192 steps");
    cudaError_t e = cudaMemsetAsync(tally, 0, sizeof(unsigned long long) * PE_PAIR_TALLY_WORDS, r->stream);
    if (e != cudaSuccess) return cuda_fail(e, "pe_bw_transport");
    if (n_photons == 0) return PE_OK;
    launch_bw_transport(bw->dev, r->dev, r->params.precision, photons, n_photons, step_end, pairs, capacity,
                        static_cast<unsigned long long*>(tally), r->stream);
    g_launches++;
    e = cudaGetLastError();
    return e == cudaSuccess ? PE_OK : cuda_fail(e, "pe_bw_transport");
}

extern "C" int pe_debug_build(void) {
#ifdef PE_DEBUG
    return 1;
#else
    return 0;
#endif
}

extern "C" pe_status pe_debug_count(const pe_tables* t, const pe_bw_tables* bw, uint64_t* out) {
    if (!out || (!t && !bw)) return fail(PE_ERR_ARG, "pe_debug_count: null argument");
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "pe_debug_count: synchronize");
    uint64_t sum = 0, v = 0;
    if (t) {
        e = cudaMemcpy(&v, t->dev.dbg, sizeof(v), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "pe_debug_count");
        sum += v;
    }
    if (bw) {
        e = cudaMemcpy(&v, bw->dev.dbg, sizeof(v), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "pe_debug_count");
        sum += v;
    }
    *out = sum;
    return PE_OK;
}

extern "C" pe_status pe_math_probe(int fn, const float* in, float* out, int64_t n, void* stream) {
    if ((n > 0 && (!in || !out)) || n < 0) return fail(PE_ERR_ARG, "pe_math_probe: null buffer or n < 0");
    if (fn < PE_MATH_RCP || fn > PE_MATH_TAU) return fail(PE_ERR_ARG, "pe_math_probe: unknown fn");
    if (n >= (int64_t(1) << 40)) return fail(PE_ERR_ARG, "pe_math_probe: n too large");
    if (n == 0) return PE_OK;
    launch_math_probe(fn, in, out, n, static_cast<cudaStream_t>(stream));
    g_launches++;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PE_OK : cuda_fail(e, "pe_math_probe");
}

extern "C" pe_status pe_fma_peak(int kind, int blocks, int threads, int iters, void* out, void* stream,
                                 int* chains_out) {
    if (kind < PE_FMA_F32 || kind > PE_FMA_F64) return fail(PE_ERR_ARG, "pe_fma_peak: unknown kind");
    if (blocks < 1 || iters < 1 || threads < 32 || threads > 256 || threads % 32 || !out)
        return fail(PE_ERR_ARG, "pe_fma_peak: need blocks, iters >= 1, threads a multiple of 32 in [32, 256], out");
    if (chains_out) *chains_out = fma_chains();
    launch_fma_peak(kind, blocks, threads, iters, out, static_cast<cudaStream_t>(stream));
    g_launches++;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PE_OK : cuda_fail(e, "pe_fma_peak");
}

extern "C" pe_status pe_destroy(pe_run* r) {
    if (!r) return fail(PE_ERR_ARG, "pe_destroy: null");
    delete r;
    return PE_OK;
}

// ---------------------------------------------------------------------------
// CUDA graph of the batched persistent launches
// ---------------------------------------------------------------------------
struct pe_graph {
    std::vector<pe_run*> runs;
    int64_t steps = 0;
    Plan plan;
    std::vector<cudaGraphNode_t> nodes;
    std::vector<cudaKernelNodeParams> params;
    std::vector<std::array<void*, 3>> args;
    std::vector<int> step_args;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t stream = nullptr;
};

extern "C" pe_status pe_graph_create(pe_run* const* runs, int n_runs, int64_t steps_per_replay,
                                     const pe_launch_config* cfg, pe_graph** out) {
    if (!out) return fail(PE_ERR_ARG, "pe_graph_create: null out");
    *out = nullptr;
    pe_status st = check_batch(runs, n_runs, steps_per_replay);
    if (st != PE_OK) return st;
    if (steps_per_replay < 1) return fail(PE_ERR_ARG, "pe_graph_create: steps_per_replay must be >= 1");
    for (int k = 0; k < n_runs; ++k)
        if (runs[k]->dev.fk == FK_PIC) return fail(PE_ERR_STATE, "pe_graph_create: PE_PIC_1D runs step through pe_step");
    pe_graph* g = new pe_graph();
    g->runs.assign(runs, runs + n_runs);
    g->steps = steps_per_replay;
    g->stream = runs[0]->stream;
    st = build_plan(runs, n_runs, steps_per_replay, cfg, g->plan);
    if (st != PE_OK) { delete g; return st; }
    const pe_tables* t = runs[0]->tables;
    cudaError_t e = cudaGraphCreate(&g->graph, 0);
    size_t nl = g->plan.launches.size();
    g->nodes.resize(nl);
    g->params.resize(nl);
    g->args.resize(nl);
    g->step_args.resize(nl);
    for (size_t k = 0; k < nl && e == cudaSuccess; ++k) {
        PlanLaunch& L = g->plan.launches[k];
        set_step0(L, runs, 0);
        g->step_args[k] = L.steps;
        void* batch = L.prec == PE_F32 ? (void*)L.bf.get() : (void*)L.bd.get();
        g->args[k] = {(void*)&t->dev, batch, (void*)&g->step_args[k]};
        cudaKernelNodeParams& p = g->params[k];
        std::memset(&p, 0, sizeof(p));
        int threads = L.block;
        int smem = L.smem;
        p.func = const_cast<void*>(L.prec == PE_F32 ? persistent_kernel_f32(*L.bf, L.steps, L.smem, L.block, &threads,
                                                                            &smem)
                                                    : persistent_kernel_f64(*L.bd, L.smem, L.block, &threads));
        p.gridDim = dim3(L.grid);
        p.blockDim = dim3(threads);
        p.sharedMemBytes = smem;
        p.kernelParams = g->args[k].data();
        e = cudaGraphAddKernelNode(&g->nodes[k], g->graph, k ? &g->nodes[k - 1] : nullptr, k ? 1 : 0, &p);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return cuda_fail(e, "pe_graph_create");
    }
    *out = g;
    return PE_OK;
}

extern "C" pe_status pe_graph_launch(pe_graph* g) {
    if (!g) return fail(PE_ERR_ARG, "pe_graph_launch: null");
    for (pe_run* r : g->runs)
        if (r->steps_done + g->steps >= (int64_t(1) << 32))
            return fail(PE_ERR_ARG, "pe_graph_launch: step index would exceed 2^32");
    cudaError_t e = cudaSuccess;
    for (size_t k = 0; k < g->plan.launches.size() && e == cudaSuccess; ++k) {
        set_step0(g->plan.launches[k], g->runs.data(), 0);
        e = cudaGraphExecKernelNodeSetParams(g->exec, g->nodes[k], &g->params[k]);
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(g->exec, g->stream);
    if (e != cudaSuccess) return cuda_fail(e, "pe_graph_launch");
    g_launches += (int64_t)g->plan.launches.size();
    for (pe_run* r : g->runs) r->steps_done += g->steps;
    return PE_OK;
}

extern "C" pe_status pe_graph_destroy(pe_graph* g) {
    if (!g) return fail(PE_ERR_ARG, "pe_graph_destroy: null");
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return PE_OK;
}

// ---------------------------------------------------------------------------
// PIC steps that allocate nothing (pe_pic_step_noalloc)
// ---------------------------------------------------------------------------
// The current sums of one PIC step and the count of CTAs done with it live in this
// fixed array instead of memory that pe_init_particles allocates: (3 x
// PE_PIC_MAX_CELLS + 1) x 8 bytes = 96 KiB + 8 bytes, held on every GPU that loads the
// library until the process exits.  All calls share it.
static __device__ __align__(256) unsigned long long g_pic_scratch[3 * PE_PIC_MAX_CELLS + 1];

namespace {

constexpr int kMaxDevices = 128;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per
// device (with that device current) and cached.  In host code the array's name
// only stands for it: kernels get this address.
pe_status pic_scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "pe_pic_step_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(PE_ERR_ARG, "pe_pic_step_noalloc: device index out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_pic_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "pe_pic_step_noalloc: cudaGetSymbolAddress of the scratch array");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return PE_OK;
}

}  // namespace

extern "C" pe_status pe_pic_step_noalloc(const pe_tables* t, const pe_run_params* rp, int64_t n,
                                         const pe_buffers* b, int64_t step0, int64_t n_steps, void* stream) {
    if (!t || !rp || !b) return fail(PE_ERR_ARG, "pe_pic_step_noalloc: null argument");
    if (rp->geometry != PE_PIC_1D) return fail(PE_ERR_ARG, "pe_pic_step_noalloc: geometry must be PE_PIC_1D");
    if (rp->n_cells < 4 || rp->n_cells > PE_PIC_MAX_CELLS)
        return fail(PE_ERR_ARG, "pe_pic_step_noalloc: n_cells must be in [4, PE_PIC_MAX_CELLS = 4096]: the fixed "
                                "scratch array holds the current sums of at most PE_PIC_MAX_CELLS cells");
    if (step0 < 0 || n_steps < 0 || step0 + n_steps >= (int64_t(1) << 32))
        return fail(PE_ERR_ARG, "pe_pic_step_noalloc: step range");
    // the same checks and the same run description as pe_init_particles
    int iz = -1;
    pe_status st = check_run(t, rp, n, b, "pe_pic_step_noalloc", &iz);
    if (st != PE_OK) return st;
    if (n == 0 || n_steps == 0) return PE_OK;
    RunDev d;
    describe_run(t, rp, n, b, iz, d);
    void* scratch = nullptr;
    st = pic_scratch_address(&scratch);
    if (st != PE_OK) return st;
    d.jacc = static_cast<unsigned long long*>(scratch);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the array keeps what the last call left: the current sums must start at zero
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * (3 * (size_t)rp->n_cells + 1), s);
    if (e != cudaSuccess) return cuda_fail(e, "pe_pic_step_noalloc: clearing the scratch array");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int64_t k = 0; k < n_steps; ++k) {
        d.step0 = step0 + k;
        launch_pic_step(t->dev, d, rp->precision, sms, s);
        g_launches += 1;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "pe_pic_step_noalloc: PIC step");
    return PE_OK;
}
