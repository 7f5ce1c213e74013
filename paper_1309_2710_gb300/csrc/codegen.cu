// codegen.cu -- f for one mechanism as straight-line FP64 code, compiled at run
// time (NVRTC) into the lane-per-cell integrator.
//
// The table-driven f reads its reaction records, efficiencies and CSR
// stoichiometry from device tables and keeps the concentrations and the
// rates of progress in per-lane arrays: about 560 loads and stores per
// evaluation for 13 species / 54 reactions. Generated for one mechanism
// (the paper's kernels were generated per mechanism too), the species
// indices, efficiencies, molar masses and net coefficients become literals,
// C_k and the production rates live in registers, and each rate of progress
// is accumulated straight into the rates of its species: only the rate
// constants, the state and the result touch memory. The arithmetic is the
// table f's (Eqs. (E:mass), (E:spec-rate), (E:rxn-rate)) in FP64, rounded
// in a different order.
//
// Scope: FP64, lane layout, at most KIN_GEN_MAX_SPECIES species and
// KIN_GEN_MAX_REACTIONS reactions (a larger f would no longer fit the
// registers); isothermal, and with the energy equation for a mechanism that
// carries cp and Hf (the rate constants then follow T inside f). NVRTC is loaded with dlopen when first needed; without it the
// generated path is unavailable and the tables serve.
#include <dlfcn.h>
#include <nvrtc.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "codegen.h"
#include "kin_embedded.h"  // the kernel sources as strings, written by the build

namespace kin {
namespace {

void appendf(std::string& s, const char* fmt, ...)
{
    va_list ap, ap2;
    va_start(ap, fmt);
    va_copy(ap2, ap);
    const int n = vsnprintf(nullptr, 0, fmt, ap);
    va_end(ap);
    if (n > 0) {
        const size_t at = s.size();
        s.resize(at + (size_t)n + 1);
        vsnprintf(&s[at], (size_t)n + 1, fmt, ap2);
        s.resize(at + (size_t)n);
    }
    va_end(ap2);
}

// Exact decimal-free literal of a double (C++17 hexadecimal floating literal).
std::string lit(double v)
{
    char b[64];
    snprintf(b, sizeof(b), "%a", v);
    return b;
}

// ------------------------------------------------------------- NVRTC ---
struct Nvrtc {
    bool ok = false;
    nvrtcResult (*create)(nvrtcProgram*, const char*, const char*, int, const char* const*, const char* const*);
    nvrtcResult (*compile)(nvrtcProgram, int, const char* const*);
    nvrtcResult (*log_size)(nvrtcProgram, size_t*);
    nvrtcResult (*log)(nvrtcProgram, char*);
    nvrtcResult (*cubin_size)(nvrtcProgram, size_t*);
    nvrtcResult (*cubin)(nvrtcProgram, char*);
    nvrtcResult (*add_name)(nvrtcProgram, const char*);
    nvrtcResult (*lowered)(nvrtcProgram, const char*, const char**);
    nvrtcResult (*destroy)(nvrtcProgram*);
    const char* (*err)(nvrtcResult);
};

Nvrtc& nvrtc()
{
    static Nvrtc n;
    static std::once_flag once;
    std::call_once(once, [] {
        const char* names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13"};
        void* h = nullptr;
        for (const char* nm : names)
            if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL))) break;
        if (!h) return;
        bool all = true;
        auto get = [&](auto& fn, const char* sym) {
            fn = reinterpret_cast<std::remove_reference_t<decltype(fn)>>(dlsym(h, sym));
            all = all && fn;
        };
        get(n.create, "nvrtcCreateProgram");
        get(n.compile, "nvrtcCompileProgram");
        get(n.log_size, "nvrtcGetProgramLogSize");
        get(n.log, "nvrtcGetProgramLog");
        get(n.cubin_size, "nvrtcGetCUBINSize");
        get(n.cubin, "nvrtcGetCUBIN");
        get(n.add_name, "nvrtcAddNameExpression");
        get(n.lowered, "nvrtcGetLoweredName");
        get(n.destroy, "nvrtcDestroyProgram");
        get(n.err, "nvrtcGetErrorString");
        n.ok = all;
    });
    return n;
}

// Fixed-width integer types for the run-time compilation (the kernel headers
// include <stdint.h> through the public header).
const char* kStdint =
    "#pragma once\n"
    "typedef signed char int8_t;\ntypedef short int16_t;\ntypedef int int32_t;\n"
    "typedef long long int64_t;\ntypedef unsigned char uint8_t;\ntypedef unsigned short uint16_t;\n"
    "typedef unsigned int uint32_t;\ntypedef unsigned long long uint64_t;\n"
    "typedef unsigned long long uintptr_t;\n#define INT32_MAX 2147483647\n";

// Kernels compiled per mechanism: the pre-pass and the persistent integrator
// for RKCK and RKC (FP64, staging 0), both register budgets, isothermal and
// (for a mechanism with thermochemistry) with the energy equation.
std::string kernel_name(bool init, int energy, int method, int occ)
{
    char b[160];
    const char* en = energy ? "true" : "false";
    if (init)
        snprintf(b, sizeof(b), "kin::init_kernel<%d, double, 0, %s, kin::GenF>", method, en);
    else
        snprintf(b, sizeof(b), "kin::integrate_kernel<%d, double, 0, %d, %s, kin::GenF>", method, occ, en);
    return b;
}

// Compiled libraries, shared by every mechanism with the same generated
// source on a device (a test suite creates the same mechanism many times).
std::mutex g_mu;
std::map<std::pair<int, std::string>, GenKernels> g_cache;

}  // namespace

bool gen_eligible(int n_species, int n_reactions)
{
    return n_species >= 1 && n_species <= KIN_GEN_MAX_SPECIES && n_reactions <= KIN_GEN_MAX_REACTIONS;
}

namespace {

// The body shared by both forms of f: mixture, rates of progress accumulated
// into the species' rates (w_i = W_i omega_i), dY/dt. Isothermal: k_j and
// k0/kinf come in K and KR. Energy: they follow x[nS] = T at every
// evaluation, as in the table f, and dT/dt closes the body.
void emit_body(std::string& s, const kin_mech_desc* d, bool energy)
{
    const int nS = d->n_species, nR = d->n_reactions;
    if (energy) {
        appendf(s, "        const double T = x[%d];\n", nS);
        s += "        const double lnT = log(T), invT = ddiv(1.0, T);\n"
             "        const double Ctot = p * 1e-6 * invT * (1.0 / R_GAS), invCtot = ddiv(1.0, Ctot);\n";
    }
    // mixture: m_k = Y_k / W_k, S = sum m_k (two partial sums), rho = Ctot / S
    for (int i = 0; i < nS; ++i) appendf(s, "        const double m%d = x[%d] * %s;\n", i, i, lit(1.0 / d->W[i]).c_str());
    std::string ev, od;
    for (int i = 0; i < nS; ++i) {
        std::string& t = (i % 2 == 0) ? ev : od;
        if (!t.empty()) t += " + ";
        appendf(t, "m%d", i);
    }
    appendf(s, "        const double S = (%s) + (%s);\n", ev.c_str(), od.empty() ? "0.0" : od.c_str());
    s += "        const double rho = Ctot * Tab<double>::inv(S);\n";
    for (int i = 0; i < nS; ++i) appendf(s, "        const double c%d = m%d * rho;\n", i, i);
    // net coefficients: which species ever change
    std::vector<char> used(nS, 0);
    std::vector<std::vector<std::pair<int, int>>> net(nR);
    for (int j = 0; j < nR; ++j) {
        int cnt[4] = {0, 0, 0, 0}, sp[4] = {-1, -1, -1, -1}, n = 0;
        auto add = [&](int k, int c) {
            if (k < 0) return;
            for (int a = 0; a < n; ++a)
                if (sp[a] == k) { cnt[a] += c; return; }
            sp[n] = k;
            cnt[n++] = c;
        };
        add(d->prod[2 * j], 1);
        add(d->prod[2 * j + 1], 1);
        add(d->reac[2 * j], -1);
        add(d->reac[2 * j + 1], -1);
        for (int a = 0; a < n; ++a)
            if (cnt[a] != 0) {
                net[j].push_back({sp[a], cnt[a]});
                used[sp[a]] = 1;
            }
    }
    for (int i = 0; i < nS; ++i)
        if (used[i]) appendf(s, "        double w%d = 0.0;\n", i);
    // Arrhenius exponent ln A + beta ln T - (Ea/R)/T with the table f's terms
    auto exponent = [&](double lnA, double beta, double Ea) {
        std::string a = lit(lnA);
        if (beta != 0.0) a += " + " + lit(beta) + " * lnT";
        if (Ea != 0.0) a += " - " + lit(Ea / R_GAS) + " * invT";
        return a;
    };
    int row = 0, fo = 0;
    for (int j = 0; j < nR; ++j) {
        const int t = d->type[j];
        appendf(s, "        {  // reaction %d\n", j);
        std::string q;
        if (energy) {
            appendf(s, "            const double a = %s;\n", exponent(d->lnA[j], d->beta[j], d->Ea[j]).c_str());
            q = "exp(a)";
        } else {
            appendf(q, "K[%d]", j);
        }
        for (int a = 0; a < 2; ++a)
            if (d->reac[2 * j + a] >= 0) appendf(q, " * c%d", d->reac[2 * j + a]);
        appendf(s, "            double q = %s;\n", q.c_str());
        if (t != KIN_RXN_PLAIN) {
            std::string a0, a1;
            int n = 0;
            for (int k = 0; k < nS; ++k) {
                const double e = d->eff[(size_t)row * nS + k];
                if (e == 0.0) continue;
                std::string& tgt = (n++ % 2 == 0) ? a0 : a1;
                if (!tgt.empty()) tgt += " + ";
                if (e == 1.0) appendf(tgt, "c%d", k);
                else appendf(tgt, "%s * c%d", lit(e).c_str(), k);
            }
            appendf(s, "            const double Mc = (%s) + (%s);\n", a0.empty() ? "0.0" : a0.c_str(),
                    a1.empty() ? "0.0" : a1.c_str());
            if (t == KIN_RXN_THIRD_BODY) {
                s += "            q *= Mc;\n";
            } else {
                if (energy)
                    appendf(s, "            const double Pr = exp((%s) - a) * Mc;\n",
                            exponent(d->lnA0[j], d->beta0[j], d->Ea0[j]).c_str());
                else
                    appendf(s, "            const double Pr = KR[%d] * Mc;\n", fo);
                s += "            q *= ddiv(Pr, 1.0 + Pr);\n";
                ++fo;
            }
            ++row;
        }
        for (auto& e : net[j])
            appendf(s, "            w%d = fma(%s, q, w%d);\n", e.first, lit(e.second * d->W[e.first]).c_str(),
                    e.first);
        s += "        }\n";
    }
    s += "        const double invrho = S * invCtot;\n";
    for (int i = 0; i < nS; ++i) {
        if (used[i]) appendf(s, "        out[%d] = w%d * invrho;\n", i, i);
        else appendf(s, "        out[%d] = 0.0;\n", i);
    }
    if (energy) {
        // sum_i H_i omega_i = sum_i (Hf_i / W_i + (cp_i / W_i)(T - T_REF)) w_i; cp = sum_i Y_i cp_i / W_i
        s += "        const double dT = T - T_REF;\n        double hw = 0.0, cpm = 0.0;\n";
        for (int i = 0; i < nS; ++i) {
            const std::string cpW = lit(d->cp[i] / d->W[i]);
            if (used[i])
                appendf(s, "        hw = fma(%s + %s * dT, w%d, hw);\n", lit(d->Hf[i] / d->W[i]).c_str(),
                        cpW.c_str(), i);
            appendf(s, "        cpm = fma(x[%d], %s, cpm);\n", i, cpW.c_str());
        }
        appendf(s, "        out[%d] = ddiv(-hw * invrho, cpm);\n", nS);
    }
}

}  // namespace

std::string gen_f_source(const kin_mech_desc* d)
{
    const int nS = d->n_species, nR = d->n_reactions;
    const bool thermo = d->cp && d->Hf;
    std::string s;
    appendf(s, "// f for one mechanism: %d species, %d reactions (generated)%s.\n", nS, nR,
            thermo ? ", isothermal and with the energy equation" : "");
    s += "namespace kin {\nstruct GenF {\n"
         "    template <typename R, typename KT>\n"
         "    __device__ __forceinline__ static void eval(const MechDev&, double Ctot, double invCtot, Lane<KT> K,\n"
         "                                                Lane<KT> KR, Lane<R>, Lane<R>, Lane<double> x,\n"
         "                                                Lane<double> out)\n    {\n"
         "        static_assert(sizeof(R) == 8 && sizeof(KT) == 8, \"the generated f is FP64\");\n";
    emit_body(s, d, false);
    s += "    }\n";
    if (thermo) {
        s += "    template <typename R>\n"
             "    __device__ __forceinline__ static void eval_energy(const MechDev&, double p, Lane<R>, Lane<R>,\n"
             "                                                       Lane<double> x, Lane<double> out)\n    {\n"
             "        static_assert(sizeof(R) == 8, \"the generated f is FP64\");\n";
        emit_body(s, d, true);
        s += "    }\n";
    }
    s += "};\n}  // namespace kin\n";
    return s;
}

int gen_compile(const std::string& f_src, std::vector<char>* cubin, std::vector<std::string>* lowered,
                std::string* log)
{
    Nvrtc& n = nvrtc();
    if (!n.ok) {
        *log = "NVRTC (libnvrtc.so.13) is not available";
        return KIN_EUNSUPPORTED;
    }
    const std::string src = std::string("#include \"kernels.cuh\"\n") + f_src;
    const char* headers[] = {kin_src_kernels, kin_src_dev, kin_src_api, kStdint};
    const char* names[] = {"kernels.cuh", "kin_dev.cuh", "../../include/kin.h", "stdint.h"};
    nvrtcProgram prog;
    nvrtcResult r = n.create(&prog, src.c_str(), "kin_generated.cu", 4, headers, names);
    if (r != NVRTC_SUCCESS) {
        *log = n.err(r);
        return KIN_ECUDA;
    }
    // per energy form: init RKCK, init RKC, integrate [method][occupancy]
    std::vector<std::string> exprs;
    const int forms = f_src.find("eval_energy") != std::string::npos ? 2 : 1;
    for (int en = 0; en < forms; ++en)
        for (int init = 1; init >= 0; --init)
            for (int method = 0; method < 2; ++method)
                for (int occ = 0; occ < (init ? 1 : 2); ++occ) exprs.push_back(kernel_name(init, en, method, occ));
    for (auto& e : exprs) n.add_name(prog, e.c_str());
    // -default-device: the public header's host declarations become (unused)
    // device declarations instead of errors
    const char* opts[] = {"--gpu-architecture=sm_103a", "--std=c++17", "-default-device"};
    r = n.compile(prog, 3, opts);
    size_t ls = 0;
    n.log_size(prog, &ls);
    std::string lg(ls, '\0');
    if (ls) n.log(prog, &lg[0]);
    *log = lg;
    if (r != NVRTC_SUCCESS) {
        n.destroy(&prog);
        return KIN_ECUDA;
    }
    size_t cs = 0;
    n.cubin_size(prog, &cs);
    cubin->assign(cs, 0);
    n.cubin(prog, cubin->data());
    lowered->clear();
    for (auto& e : exprs) {
        const char* ln = nullptr;
        n.lowered(prog, e.c_str(), &ln);
        lowered->push_back(ln ? ln : "");
    }
    n.destroy(&prog);
    return KIN_OK;
}

int gen_kernels(int device, const std::string& f_src, GenKernels* out, std::string* log)
{
    std::lock_guard<std::mutex> lk(g_mu);
    auto key = std::make_pair(device, f_src);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
        *out = it->second;
        return KIN_OK;
    }
    std::vector<char> cubin;
    std::vector<std::string> names;
    int rc = gen_compile(f_src, &cubin, &names, log);
    if (rc != KIN_OK) return rc;
    GenKernels g{};
    cudaError_t e = cudaLibraryLoadData(&g.lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e != cudaSuccess) {
        *log = cudaGetErrorString(e);
        cudaGetLastError();
        return KIN_ECUDA;
    }
    // names per energy form: init RKCK, init RKC, then integrate [method][occ]
    g.energy = names.size() == 12;
    e = cudaSuccess;
    for (int en = 0; en < (g.energy ? 2 : 1) && e == cudaSuccess; ++en) {
        const int b = 6 * en;
        e = cudaLibraryGetKernel(&g.init[en][0], g.lib, names[b].c_str());
        if (e == cudaSuccess) e = cudaLibraryGetKernel(&g.init[en][1], g.lib, names[b + 1].c_str());
        for (int k = 0; k < 4 && e == cudaSuccess; ++k)
            e = cudaLibraryGetKernel(&g.integrate[en][k / 2][k % 2], g.lib, names[b + 2 + k].c_str());
    }
    if (e != cudaSuccess) {
        *log = cudaGetErrorString(e);
        cudaGetLastError();
        cudaLibraryUnload(g.lib);
        return KIN_ECUDA;
    }
    g_cache[key] = g;
    *out = g;
    return KIN_OK;
}

bool gen_loaded(int device, const std::string& f_src)
{
    std::lock_guard<std::mutex> lk(g_mu);
    return g_cache.count(std::make_pair(device, f_src)) > 0;
}

cudaError_t gen_launch(const GenKernels& g, Launch& L, int occ, int blocks, int threads, cudaStream_t st)
{
    if (L.energy && !g.energy) return cudaErrorInvalidValue;  // refused by the caller before
    void* args[] = {&L};
    const int m = L.method == KIN_RKC ? 1 : 0, en = L.energy ? 1 : 0;
    cudaError_t e = cudaLaunchKernel((const void*)g.init[en][m], dim3(blocks), dim3(threads), args, 0, st);
    if (e != cudaSuccess) return e;
    if (L.method == KIN_RKC) {
        e = launch_sort(L, st);
        if (e != cudaSuccess) return e;
    }
    return cudaLaunchKernel((const void*)g.integrate[en][m][occ ? 1 : 0], dim3(blocks), dim3(threads), args, 0,
                            st);
}

}  // namespace kin
