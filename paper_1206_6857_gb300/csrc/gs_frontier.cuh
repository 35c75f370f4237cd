// Frontier data structures shared by the traversal, series and base-case
// kernels.
#pragma once

#include <stdint.h>

namespace gs {

// Pair actions (one per frontier pair and iteration).
enum : int { M_FD = 0, M_DH = 1, M_DL = 2, M_H2L = 3, M_BASE = 4, M_SPLIT = 5 };

// A group is every frontier pair sharing one query node and one bandwidth;
// its pairs' reference nodes are stored contiguously (ascending) at off.
struct Group {
    int32_t q, j;
    int64_t off;
    int32_t cnt, pad;
};

// One series action: method M_DH / M_DL / M_H2L at order p.
struct SeriesEntry {
    int32_t q, r;
    int16_t j;
    int8_t p, method;
    int32_t pad;
};

// per-group counts: child pairs, child groups, base pairs, DH, DL, H2L actions, base groups
constexpr int kCols = 7;
enum : int { C_PAIRS = 0, C_GROUPS = 1, C_BASE = 2, C_DH = 3, C_DL = 4, C_H2L = 5, C_BGROUPS = 6 };

// Device-resident traversal bookkeeping (one instance per call).
struct FrontierState {
    int64_t ngroups[72];        // groups in iteration t
    int64_t npairs[72];         // pairs in iteration t
    int64_t base_count, base_groups, trace_count;
    int64_t series_count[3];    // DH, DL, H2L actions so far
    int64_t totals[kCols];      // column totals of the last scan
    unsigned long long method_count[6];
    double eps_t, rho, Wtot, floorW;
    unsigned long long work;    // tile counter of dynamically scheduled kernels (zeroed before each)
    double diam;                // diagonal of the reference root box
    int32_t overflow;
    int32_t pad;
};

}  // namespace gs
