// tables.cu -- class tables of the triad counters, built on the host from the
// definitions of paper Section II and uploaded once per process.
//
// A Venn region of an ordered triple (a,b,c) is named here by a 3-bit code of
// the sets holding it (a = 1, b = 2, c = 4).  Region bit r of a pattern:
//   r:    0   1   2   3    4    5    6
//   code: a   b   c   ab   bc   ac   abc
// A pattern is a triad pattern when all three sets are non-empty and at
// least two of the three pairs share a region (connected triple).
#include <algorithm>
#include <vector>

#include "escher_internal.cuh"

namespace esc {

namespace {

const int kCodeOfRegion[7] = {1, 2, 4, 3, 6, 5, 7};

int region_of_code(int code) {
    for (int r = 0; r < 7; ++r)
        if (kCodeOfRegion[r] == code) return r;
    return -1;
}

bool nonempty(int mask, int set_bit) {
    for (int r = 0; r < 7; ++r)
        if ((mask >> r & 1) && (kCodeOfRegion[r] & set_bit)) return true;
    return false;
}

bool pair_meets(int mask, int pair_bits) {
    for (int r = 0; r < 7; ++r)
        if ((mask >> r & 1) && (kCodeOfRegion[r] & pair_bits) == pair_bits) return true;
    return false;
}

// two sets are identical when no region holds exactly one of them
bool pair_identical(int mask, int s, int t) {
    for (int r = 0; r < 7; ++r) {
        if (!(mask >> r & 1)) continue;
        int c = kCodeOfRegion[r];
        if (((c & s) != 0) != ((c & t) != 0)) return false;
    }
    return true;
}

bool is_triad(int mask) {
    if (!nonempty(mask, 1) || !nonempty(mask, 2) || !nonempty(mask, 4)) return false;
    return int(pair_meets(mask, 3)) + int(pair_meets(mask, 6)) + int(pair_meets(mask, 5)) >= 2;
}

// orders of the labels: new label k is old label kOrder[q][k]
const int kOrder[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

int reorder(int mask, int q) {
    int out = 0;
    for (int r = 0; r < 7; ++r) {
        if (!(mask >> r & 1)) continue;
        int c = kCodeOfRegion[r], nc = 0;
        for (int k = 0; k < 3; ++k)
            if (c >> kOrder[q][k] & 1) nc |= 1 << k;
        out |= 1 << region_of_code(nc);
    }
    return out;
}

}  // namespace

void build_class_tables(ClassTables* t) {
    std::vector<int> reps_plain, reps_twin, valid;
    for (int m = 0; m < 128; ++m) {
        for (int q = 0; q < 6; ++q) t->perm[q][m] = uint8_t(reorder(m, q));
        t->cls30[m] = -1;
        t->cls96[m] = -1;
    }
    for (int m = 0; m < 128; ++m) {
        if (!is_triad(m)) continue;
        valid.push_back(m);
        int lo = m;
        for (int q = 0; q < 6; ++q) lo = std::min(lo, reorder(m, q));
        if (lo != m) continue;
        bool twin = pair_identical(m, 1, 2) || pair_identical(m, 2, 4) || pair_identical(m, 1, 4);
        (twin ? reps_twin : reps_plain).push_back(m);
    }
    std::vector<int> reps = reps_plain;  // ascending: masks were visited in order
    reps.insert(reps.end(), reps_twin.begin(), reps_twin.end());
    for (int m : valid) {
        int lo = m;
        for (int q = 0; q < 6; ++q) lo = std::min(lo, reorder(m, q));
        t->cls30[m] = int8_t(std::find(reps.begin(), reps.end(), lo) - reps.begin());
    }
    for (size_t i = 0; i < valid.size(); ++i) t->cls96[valid[i]] = int8_t(i);
}

}  // namespace esc
