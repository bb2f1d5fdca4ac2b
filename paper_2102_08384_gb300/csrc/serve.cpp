// Serving loop (continuous batching of estimator requests); see bym.h.
#include "engine.h"

namespace bym {

void shutdown_serving(bym_ctx *c) { (void)c; }

}  // namespace bym
