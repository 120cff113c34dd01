/* A plain C99 caller of the library's host-only entry points: the header is
 * C, the library links from C, and the calls need no GPU.  Prints one line
 * per check; the pytest wrapper compares them. */
#include <stdint.h>
#include <stdio.h>

#include "pac.h"

int main(void) {
    int radices[64];
    int count = 64;
    if (pac_stage_list(1000, 0, radices, &count) != PAC_OK) return 1;
    printf("stages");
    for (int i = 0; i < count; ++i) printf(" %d", radices[i]);
    printf("\n");

    int stages[3] = {4, 4, 2};
    int64_t p2f[32];
    if (pac_reverse_table(3, stages, p2f) != PAC_OK) return 2;
    printf("reverse %lld %lld %lld\n", (long long)p2f[0], (long long)p2f[1], (long long)p2f[31]);

    int64_t dims[3] = {6000, 1, 1};
    int axis[8], size[8], rounds[64], ng = 8;
    if (pac_plan_groups(1, dims, 0, PAC_C64, 1, 0, axis, size, rounds, &ng) != PAC_OK) return 3;
    printf("groups %d", ng);
    for (int g = 0; g < ng; ++g) printf(" %d", size[g]);
    printf("\n");

    int rc = pac_stage_list(7, 0, radices, &count);
    printf("error %d %s\n", rc, pac_last_error()[0] ? "message" : "none");
    printf("version %s\n", pac_version());
    return 0;
}
