// Serving scheduler placeholder: no jobs are ever queued yet.
#include "internal.h"

namespace grav {
void serve_shutdown(grav_ctx *) {}
}  // namespace grav
