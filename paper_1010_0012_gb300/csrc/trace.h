// Tracing and logging of the library's calls.  Every traced entry point opens
// an NVTX range named after itself (visible to profilers that record NVTX
// ranges; free when none listens).  When the environment variable BP_LOG is
// set to a value other than 0 at the first traced call, each traced call also
// writes one line to stderr with its host-side time, and every error a call
// reports is written with its status and message.  Internal.
#pragma once

#include <nvtx3/nvToolsExt.h>

#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <string>

namespace bpg {

inline bool log_enabled() {
    static const bool on = [] {
        const char *v = std::getenv("BP_LOG");
        return v && *v && !(v[0] == '0' && v[1] == 0);
    }();
    return on;
}

inline void log_error(int status, const std::string &msg) {
    if (log_enabled()) std::fprintf(stderr, "[bp] error %d: %s\n", status, msg.c_str());
}

class ApiScope {
  public:
    explicit ApiScope(const char *name) : name_(name) {
        nvtxRangePushA(name);
        if (log_enabled()) t0_ = std::chrono::steady_clock::now();
    }
    ~ApiScope() {
        nvtxRangePop();
        if (log_enabled()) {
            const double us =
                std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0_).count();
            std::fprintf(stderr, "[bp] %s %.1f us host\n", name_, us);
        }
    }
    ApiScope(const ApiScope &) = delete;
    ApiScope &operator=(const ApiScope &) = delete;

  private:
    const char *name_;
    std::chrono::steady_clock::time_point t0_{};
};

}  // namespace bpg

#define BPG_TRACE(name) bpg::ApiScope bpg_trace_scope_(name)
