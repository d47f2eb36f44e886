#include <algorithm>
#include <type_traits>
#define BCG_T float
#include "bcg_stream.inc"
