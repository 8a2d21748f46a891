// mg.cu -- geometric multigrid hierarchy and V-cycle (internal).
#include "mg.h"

namespace stokes {

struct MgHierarchy {
    bool stale = true;
};

void mg_invalidate(MgHierarchy *h)
{
    if (h) h->stale = true;
}

void mg_destroy(MgHierarchy *h) { delete h; }

} // namespace stokes
