#include <algorithm>
#include <type_traits>
#define BCG_T double
#include "bcg_stream.inc"
