// mg.h -- geometric multigrid hierarchy of a context (internal).
#pragma once

namespace stokes {

struct MgHierarchy;

// Mark the hierarchy stale (the viscosity changed); the next solve rebuilds it.
void mg_invalidate(MgHierarchy *h);
// Free every buffer of the hierarchy.  Accepts NULL.
void mg_destroy(MgHierarchy *h);

} // namespace stokes
