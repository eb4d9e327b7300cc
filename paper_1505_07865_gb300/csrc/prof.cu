// Launch counting and optional per-launch CUDA-event timing of every kernel
// class of the library, with the algorithmic bytes each launch must move
// (each array read or written once).  Process-wide; intended for one host
// thread driving the library at a time.
#include <atomic>
#include <cstring>
#include <string>
#include <mutex>
#include <vector>

#include <cstdlib>

#include "ibr_internal.cuh"

namespace ibr {

static std::atomic<long long> g_launches{0};
static bool g_prof = false;

bool pdl_enabled() {
    static const bool on = [] {
        const char* e = std::getenv("IBR_PDL");
        return !(e && e[0] == '0');
    }();
    return on;
}

struct Pending {
    int kid;
    cudaEvent_t a, b;
    double bytes, flops;
    int count;
};
struct Acc {
    long long launches = 0;
    double ms = 0.0;
    double bytes = 0.0;
    double flops = 0.0;
};
static std::mutex g_mu;
static std::vector<Pending> g_pending;
static std::vector<cudaEvent_t> g_free;
// [0, KID_COUNT): all launches of a class; [KID_COUNT, 2 KID_COUNT): only its
// launches that move >= kLargeBytes (the HBM-bound ones)
constexpr double kLargeBytes = 32.0 * 1024 * 1024;
static Acc g_acc[2 * KID_COUNT];

static const char* kNames[KID_COUNT] = {
    "stokes_apply", "mg_smooth_rbgs", "mg_residual_restrict", "mg_prolong_correct", "mg_coarse_solve",
    "ps_divergence", "ps_finish", "vec_axpby", "vec_scale_copy", "vec_convert", "krylov_mdot",
    "krylov_update_mdot", "krylov_update_norm2", "krylov_norm2", "krylov_combine", "block_means",
    "subtract_means", "krylov_small", "spread_gather", "interp", "lam_sum", "rigid_K", "rigid_KT",
    "markers_setup", "mtilde_build", "spd_inverse", "blockdiag_gemv", "advect", "tc_gemm_tf32x3",
};

// per-thread count as well: a graph capture counts only its own thread's launches
static thread_local long long t_launches = 0;
void count_launch() {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    ++t_launches;
}
void add_launches(long long n) {
    g_launches.fetch_add(n, std::memory_order_relaxed);
    t_launches += n;
}
long long thread_launches() { return t_launches; }
bool profiling_enabled() { return g_prof; }

static cudaEvent_t get_event() {
    if (!g_free.empty()) {
        cudaEvent_t e = g_free.back();
        g_free.pop_back();
        return e;
    }
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

ProfScope::ProfScope(int kid, cudaStream_t s, double bytes, double flops, int count)
    : kid_(kid), s_(s), bytes_(bytes), flops_(flops), count_(count), a_(nullptr) {
    if (!g_prof) return;
    std::lock_guard<std::mutex> lk(g_mu);
    a_ = get_event();
    if (a_) cudaEventRecord((cudaEvent_t)a_, s_);
}

ProfScope::~ProfScope() {
    if (!a_) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t b = get_event();
    if (!b) return;
    cudaEventRecord(b, s_);
    g_pending.push_back({kid_, (cudaEvent_t)a_, b, bytes_, flops_, count_});
}

static void drain() {
    for (auto& p : g_pending) {
        cudaEventSynchronize(p.b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, p.a, p.b);
        for (int q = 0; q < 2; ++q) {
            if (q == 1 && p.bytes < kLargeBytes * p.count) break;
            Acc& a = g_acc[p.kid + q * KID_COUNT];
            a.launches += p.count;
            a.ms += ms;
            a.bytes += p.bytes;
            a.flops += p.flops;
        }
        g_free.push_back(p.a);
        g_free.push_back(p.b);
    }
    g_pending.clear();
}

}  // namespace ibr

extern "C" {

int ibr_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(ibr::g_mu);
    ibr::g_prof = on != 0;
    return IBR_OK;
}

int ibr_profile_reset(void) {
    std::lock_guard<std::mutex> lk(ibr::g_mu);
    ibr::drain();
    for (auto& a : ibr::g_acc) a = ibr::Acc();
    return IBR_OK;
}

int ibr_profile_read(int idx, char* name, int name_len, long long* launches, double* ms, double* bytes,
                     double* flops) {
    if (idx < 0 || idx >= 2 * ibr::KID_COUNT) return IBR_EINVAL;
    std::lock_guard<std::mutex> lk(ibr::g_mu);
    ibr::drain();
    const ibr::Acc& a = ibr::g_acc[idx];
    if (name && name_len > 0) {
        std::string nm = ibr::kNames[idx % ibr::KID_COUNT];
        if (idx >= ibr::KID_COUNT) nm += "@large";
        std::strncpy(name, nm.c_str(), (size_t)name_len - 1);
        name[name_len - 1] = 0;
    }
    if (launches) *launches = a.launches;
    if (ms) *ms = a.ms;
    if (bytes) *bytes = a.bytes;
    if (flops) *flops = a.flops;
    return IBR_OK;
}

long long ibr_launch_count(void) { return ibr::g_launches.load(); }

}  // extern "C"
