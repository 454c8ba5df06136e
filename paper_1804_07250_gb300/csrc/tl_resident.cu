// Placeholder translation unit for the shared-memory resident kernel.
#include "tl_internal.h"
