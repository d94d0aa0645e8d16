/* Uses libcow from plain C (no C++, no Python): the header compiles as C and
 * the host-only calls work without a GPU.  Built and run by test_abi.py. */
#include <stdio.h>
#include <string.h>

#include "cow.h"

int main(void) {
    if (cow_version() != 1) return 1;
    /* views A = {0, 1}, B = {2, 3}, C = {0, 1}; room for two blocks of 10 bytes */
    const int64_t bytes[4] = {10, 10, 10, 10};
    const int32_t ids[6] = {0, 1, 2, 3, 0, 1};
    const int32_t offs[4] = {0, 2, 4, 6};
    int32_t order[3];
    int64_t planned = -1, given = -1;
    if (cow_plan_view_order(bytes, 4, ids, offs, 3, 20, order, &planned, &given) != COW_OK) return 2;
    if (planned != 40 || given != 60 || order[0] != 0 || order[1] != 2 || order[2] != 1) return 3;
    /* a view over the budget is rejected with a message */
    if (cow_plan_view_order(bytes, 4, ids, offs, 3, 15, order, NULL, NULL) != COW_ERR_INVALID_ARG) return 4;
    if (strlen(cow_last_error()) == 0) return 5;
    if (cow_set_schedule(NULL, COW_SCHED_THREAD_CONST) != COW_ERR_INVALID_ARG) return 6;
    printf("ok %d %lld %lld\n", (int)COW_SCHED_THREAD_CONST, (long long)planned, (long long)given);
    return 0;
}
