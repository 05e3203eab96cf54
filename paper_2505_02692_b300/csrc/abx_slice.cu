// Frame slicing by onset / offset (fastabx App. A).  Frame i stands for time
// t_i = dt/2 + i dt; a unit [t_on, t_off] keeps the frames with
// t_on <= t_i <= t_off, i.e. (Eqs. 3-4)
//   first = ceil(t_on / dt - 1/2),   last = floor(t_off / dt - 1/2),
// both included.  The Libri-Light convention keeps last - 1 instead of last.
// Times are integers in one unit, so the bounds are exact:
//   first = ceil((2 t_on - dt) / (2 dt)),  last = floor((2 t_off - dt) / (2 dt)).
#include <stdint.h>

#include "abx_internal.h"

namespace {

int64_t ceil_div(int64_t a, int64_t b) { return a >= 0 ? (a + b - 1) / b : -((-a) / b); }
int64_t floor_div(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

bool slice_one(int64_t t_on, int64_t t_off, int64_t dt, int32_t libri_light, int64_t *first,
               int64_t *last) {
    if (dt <= 0 || t_on < 0 || t_off < t_on) return false;
    int64_t a = ceil_div(2 * t_on - dt, 2 * dt);
    if (a < 0) a = 0;
    int64_t b = floor_div(2 * t_off - dt, 2 * dt);
    if (libri_light && b >= a) b -= 1;
    *first = a;
    *last = b;
    return true;
}

}  // namespace

extern "C" int abx_slice_frames(int64_t t_on, int64_t t_off, int64_t dt, int32_t libri_light,
                                int64_t *first, int64_t *last) {
    if (!first || !last || !slice_one(t_on, t_off, dt, libri_light, first, last)) {
        abx::set_error("abx_slice_frames: need dt > 0, 0 <= t_on <= t_off, non-NULL outputs");
        return ABX_E_INVALID;
    }
    return ABX_OK;
}

extern "C" int abx_slice_items(int64_t n, const int64_t *t_on, const int64_t *t_off, int64_t dt,
                               int32_t libri_light, int64_t *first, int64_t *last) {
    if (n < 0 || (n > 0 && (!t_on || !t_off || !first || !last))) {
        abx::set_error("abx_slice_items: NULL argument");
        return ABX_E_INVALID;
    }
    for (int64_t k = 0; k < n; ++k)
        if (!slice_one(t_on[k], t_off[k], dt, libri_light, &first[k], &last[k])) {
            abx::set_error("abx_slice_items: item %lld has bad times", (long long)k);
            return ABX_E_INVALID;
        }
    return ABX_OK;
}
