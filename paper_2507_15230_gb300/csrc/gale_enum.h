// The enumeration as the coboundary pass reads it, and the device
// enumeration the host side calls (internal).
#pragma once

#include <stdint.h>

#include <vector>

#include "gale_ctx.h"
#include "gale_par.h"

namespace gale {

// Host arrays of the current enumeration (gale_enum.cpp), valid while the
// context holds it.  ebk / fbk are null when ids follow the vertex-tuple
// order (the lexicographic numbering); E / F are null while the lists exist
// only on the device (device_enumeration).
struct EnumView {
    int32_t order;
    uint64_t gen;
    int32_t K;
    int64_t nE, nF;
    const int32_t *E, *F, *ebk, *fbk;
    const int64_t *IE, *IF;
};
bool enumeration_view(gale_ctx *ctx, EnumView *v);

// Sorted enumeration on the device (gale_cobound.cu): I_E and I_F into
// host vectors; the lists E and F stay on the device with the coboundary
// pass, tagged with gen.  Builds the ET rows of every cluster first.
// ENOTFOUND (nothing done) when the context cannot: no device or ET not
// preconditioned.
gale_status enumerate_sorted_device(gale_ctx *ctx, uint64_t gen, std::vector<int64_t> &IE,
                                    std::vector<int64_t> &IF);

// Device copies of enumeration gen's lists E [2 nE] and F [3 nF], if the
// coboundary pass holds them (gale_cobound.cu).
bool device_enumeration(gale_ctx *ctx, uint64_t gen, const int32_t **E, const int32_t **F);

}  // namespace gale
