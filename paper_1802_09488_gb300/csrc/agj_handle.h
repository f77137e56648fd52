// agj_handle.h — the opaque handle behind agj_index (include/agj.h), shared
// by the translation units that implement the C ABI.
#pragma once

#include "agj_index.h"

struct agj_index {
    agj::Index X;
};
