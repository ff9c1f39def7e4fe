/*
 * K-sort oracle (arxiv 1107.3622, Section 1.1). TEST INFRASTRUCTURE ONLY: see
 * ksort_ref.h for who may use it. The algorithm body lives in ksort_ref_body.h and
 * is instantiated here once per element type.
 */
#include <stdlib.h>
#include <string.h>

#include "ksort_ref.h"

#define KT float
#define KNAME(x) x##_f32
#include "ksort_ref_body.h"
#undef KT
#undef KNAME

#define KT double
#define KNAME(x) x##_f64
#include "ksort_ref_body.h"
#undef KT
#undef KNAME

#define KT uint32_t
#define KNAME(x) x##_u32
#include "ksort_ref_body.h"
#undef KT
#undef KNAME
