/* Plain C client of the library (no GPU needed): it includes both public
 * headers, links against the shared library, and exercises the entry points'
 * argument checks and the error reporting, which run on the host before any
 * device work.  Prints "ok" or the first unexpected status. */
#include <stdio.h>
#include <string.h>

#include "xorgens_gb300.h"
#include "xorgens_w64.h"

static int expect(const char* what, xg_status got, xg_status want)
{
    if (got != want) {
        printf("FAIL %s: status %d, expected %d (%s)\n", what, (int)got, (int)want, xg_last_error());
        return 1;
    }
    return 0;
}

int main(void)
{
    int bad = 0;
    uint32_t v[6];
    uint64_t omega = 0;
    bad |= expect("create with null handle", xg_create_streams(NULL, 4, 0, 1, NULL), XG_EINVAL);
    bad |= expect("generate on null context", xg_generate_u32(NULL, 0, 1, 8, NULL, 8), XG_EINVAL);
    if (strlen(xg_last_error()) == 0) {
        printf("FAIL: empty error message\n");
        bad = 1;
    }
    bad |= expect("seed on null context", xg_seed(NULL, 0, 1, NULL), XG_EINVAL);
    bad |= expect("submit on null context", xg_submit(NULL, NULL, NULL), XG_EINVAL);
    bad |= expect("destroy null", xg_destroy(NULL), XG_OK);
    bad |= expect("w64 params", xg_w64_params(v, &omega), XG_OK);
    if (v[0] != 64 || omega != 0x9E3779B97F4A7C15ull) {
        printf("FAIL: w64 params %u %llx\n", v[0], (unsigned long long)omega);
        bad = 1;
    }
    bad |= expect("w64 create with null handle", xg_w64_create(NULL, 4, 1, NULL), XG_EINVAL);
    bad |= expect("w64 destroy null", xg_w64_destroy(NULL), XG_OK);
    if (strstr(xg_version(), "sm_103a") == NULL) {
        printf("FAIL: version %s\n", xg_version());
        bad = 1;
    }
    if (!bad) printf("ok\n");
    return bad;
}
