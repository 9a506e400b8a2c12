// conflict_ubsan_main.cpp -- the conflict detector (conflict.cpp) built on its
// own, with the undefined-behaviour sanitizer, and run over every mode and
// shared-state pattern with the host-timer offload, with and without store
// emulation, plus its store self-test.  The served-path calls it can make are
// stubbed (this build has no GPU path): a run with srv == NULL never makes them.
#include "aesoffload.h"

#include <cstdio>

extern "C" {
int offload_submit(offload_server_t, int, const uint8_t *, const void *, void *, size_t, uint64_t *)
{
    return AES_EINVAL;
}
int offload_submit_emulated(offload_server_t, uint64_t, uint64_t *) { return AES_EINVAL; }
int offload_poll(offload_server_t, uint64_t) { return AES_EINVAL; }
}

int main()
{
    int bad = 0;
    for (int emu = 0; emu < 2; ++emu)
        for (int mode = CDET_UNPROTECTED; mode <= CDET_ENFORCE; ++mode)
            for (int pat = CDET_PATTERN_SHARED; pat <= CDET_PATTERN_LOCKED; ++pat) {
                cdet_run_cfg_t c{};
                c.handlers = 16;
                c.requests = 1500;
                c.counters = 64;
                c.counters_per_page = 1;
                c.mode = mode;
                c.offload_ns = 20000;
                c.pattern = pat;
                c.store_mode = emu ? CDET_STORES_EMULATE : CDET_STORES_UNPROTECT;
                cdet_run_result_t r{};
                const int rc = cdet_run(&c, &r);
                const bool lost_ok = mode == CDET_UNPROTECTED || mode == CDET_DETECT ? true : r.lost_updates == 0;
                if (rc || !lost_ok || (pat != CDET_PATTERN_SHARED && r.conflicts)) {
                    ++bad;
                    std::printf("bad: emulate=%d mode=%d pattern=%d rc=%d lost=%llu conflicts=%llu\n", emu, mode,
                                pat, rc, (unsigned long long)r.lost_updates, (unsigned long long)r.conflicts);
                }
            }
    uint64_t emulated = 0, fallbacks = 0;
    const int rc = cdet_store_selftest(9000, &emulated, &fallbacks);
    std::printf("%s selftest rc=%d emulated=%llu fallbacks=%llu\n", bad || rc ? "FAIL" : "OK", rc,
                (unsigned long long)emulated, (unsigned long long)fallbacks);
    return bad || rc ? 1 : 0;
}
