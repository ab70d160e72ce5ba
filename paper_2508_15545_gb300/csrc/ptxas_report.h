// Reading the ptxas -v report NVRTC returns for a compiled pass (host only):
// the register count and whether any function of the module spills.
#pragma once

#include <cstdlib>
#include <string>

namespace qv {

// The number in front of every occurrence of `key` ("Used 128 registers",
// "44 bytes spill stores"): the largest (`largest`) or whether any is nonzero
// (returned as 1 / 0); -1 when `key` never occurs.
inline long ptxas_scan(const std::string &log, const char *key, bool largest)
{
    long best = -1;
    for (size_t p = log.find(key); p != std::string::npos; p = log.find(key, p + 1)) {
        size_t e = p;
        while (e > 0 && log[e - 1] == ' ') --e;
        size_t b = e;
        while (b > 0 && log[b - 1] >= '0' && log[b - 1] <= '9') --b;
        if (b == e) continue;
        const long v = std::atol(log.c_str() + b);
        if (largest) best = v > best ? v : best;
        else best = (best > 0 || v > 0) ? 1 : 0;
    }
    return best;
}

inline long ptxas_registers(const std::string &log) { return ptxas_scan(log, "registers", true); }
inline bool ptxas_spills(const std::string &log) { return ptxas_scan(log, "bytes spill stores", false) > 0; }

}  // namespace qv
