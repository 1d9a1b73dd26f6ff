// Optional per-kernel CUDA-event timing of library launches (off by default),
// with the algorithmic bytes each launch must move (inputs read once plus
// outputs written once, as counted by the launch site).
// When enabled, each instrumented launch is bracketed by two events on its
// own stream; elapsed times are accumulated lazily when the pending list is
// flushed (on read, or when it grows large).
#include <vector>

#include "common.cuh"

namespace vie {

namespace {
struct Pending {
    int id;
    cudaEvent_t a, b;
    double bytes;
};
struct TimerState {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    std::vector<Pending> pending;
    cudaEvent_t open_ev[TMR_COUNT] = {};
    double ms[TMR_COUNT] = {};
    long long cnt[TMR_COUNT] = {};
    double bytes[TMR_COUNT] = {};
};
TimerState& T() {
    static TimerState t;
    return t;
}
cudaEvent_t get_event() {
    TimerState& t = T();
    if (!t.pool.empty()) {
        cudaEvent_t e = t.pool.back();
        t.pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
void flush() {
    TimerState& t = T();
    for (Pending& p : t.pending) {
        cudaEventSynchronize(p.b);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            t.ms[p.id] += ms;
            t.cnt[p.id] += 1;
            t.bytes[p.id] += p.bytes;
        }
        t.pool.push_back(p.a);
        t.pool.push_back(p.b);
    }
    t.pending.clear();
}
const char* kNames[TMR_COUNT] = {"zfwd", "yfwd", "xfused", "yinv", "zinv", "dots", "reduce_dots", "update",
                                 "finish", "scale", "xupdate", "residual", "start_cycle", "rhs", "other",
                                 "matvec_fp64", "reorth_steps", "matvec_f32x2", "sweep", "farfield_gemm", "farfield_other"};
}  // namespace

bool tmr_enabled() { return T().on; }

void tmr_add(int id, double bytes, long long count) {
    TimerState& t = T();
    if (!t.on) return;
    t.bytes[id] += bytes;
    t.cnt[id] += count;
}

void tmr_begin(int id, cudaStream_t s) {
    TimerState& t = T();
    if (!t.on) return;
    cudaEvent_t e = get_event();
    cudaEventRecord(e, s);
    t.open_ev[id] = e;
}

void tmr_end(int id, cudaStream_t s, double bytes) {
    TimerState& t = T();
    if (!t.on || !t.open_ev[id]) return;
    cudaEvent_t e = get_event();
    cudaEventRecord(e, s);
    t.pending.push_back({id, t.open_ev[id], e, bytes});
    t.open_ev[id] = nullptr;
    if (t.pending.size() > 4096) flush();
}

}  // namespace vie

extern "C" {

void vie_timer_enable(int on) {
    vie::TimerState& t = vie::T();
    if (!on) vie::flush();
    t.on = on != 0;
}

void vie_timer_reset(void) {
    vie::flush();
    vie::TimerState& t = vie::T();
    for (int i = 0; i < vie::TMR_COUNT; ++i) {
        t.ms[i] = 0;
        t.cnt[i] = 0;
        t.bytes[i] = 0;
    }
}

int vie_timer_read(int id, double* total_ms, long long* launches, double* bytes) {
    if (id < 0 || id >= vie::TMR_COUNT) return VIE_EINVAL;
    vie::flush();
    vie::TimerState& t = vie::T();
    if (total_ms) *total_ms = t.ms[id];
    if (launches) *launches = t.cnt[id];
    if (bytes) *bytes = t.bytes[id];
    return VIE_OK;
}

const char* vie_timer_name(int id) {
    if (id < 0 || id >= vie::TMR_COUNT) return "";
    return vie::kNames[id];
}

int vie_timer_count(void) { return vie::TMR_COUNT; }

}  // extern "C"
