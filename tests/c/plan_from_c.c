/* The C-ABI used from plain C (no C++, no Python): reads a block-loss grid
 * in the golden-file format ("grid H W", then H rows of group indices, -1 =
 * no loss) from standard input, plans it with fse_plan_order in the order
 * given as the first argument (0 line scan, 1 Algorithm 1 of Sec. 3), and
 * prints the resulting grid in the same format.  Also checks the error
 * paths that need no GPU.  Exit status 0 on success. */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "fse.h"

int main(int argc, char **argv) {
    int order = argc > 1 ? atoi(argv[1]) : 1;
    char word[16];
    int bh = 0, bw = 0;
    if (scanf("%15s %d %d", word, &bh, &bw) != 3 || strcmp(word, "grid") != 0 || bh <= 0 ||
        bw <= 0)
        return 2;
    const int nb = bh * bw;
    uint8_t *lost = malloc((size_t)nb);
    int32_t *gob = malloc(sizeof(int32_t) * (size_t)nb);
    int32_t *gptr = malloc(sizeof(int32_t) * (size_t)(nb + 1));
    int32_t *ids = malloc(sizeof(int32_t) * (size_t)nb);
    if (!lost || !gob || !gptr || !ids) return 3;
    for (int i = 0; i < nb; ++i) {
        int g = 0;
        if (scanf("%d", &g) != 1) return 2;
        lost[i] = (uint8_t)(g >= 0);
    }
    int32_t ng = -1;
    int rc = fse_plan_order(bw, bh, lost, order, gob, gptr, ids, &ng);
    if (rc != FSE_OK) {
        fprintf(stderr, "fse_plan_order: %s\n", fse_strerror(rc));
        return 4;
    }
    /* every group lists its blocks in raster order and agrees with gob */
    for (int32_t g = 0; g < ng; ++g) {
        if (gptr[g + 1] <= gptr[g]) return 5;
        for (int32_t j = gptr[g]; j < gptr[g + 1]; ++j) {
            if (gob[ids[j]] != g) return 5;
            if (j > gptr[g] && ids[j] <= ids[j - 1]) return 5;
        }
    }
    /* error paths: bad order, NULL output, non-positive sizes */
    if (fse_plan_order(bw, bh, lost, 7, gob, gptr, ids, &ng) != FSE_EINVAL) return 6;
    if (fse_plan_order(bw, bh, lost, order, NULL, gptr, ids, &ng) != FSE_EINVAL) return 6;
    if (fse_plan_order(0, bh, lost, order, gob, gptr, ids, &ng) != FSE_EINVAL) return 6;
    if (strcmp(fse_strerror(FSE_OK), "ok") != 0) return 7;
    printf("grid %d %d\n", bh, bw);
    for (int y = 0; y < bh; ++y) {
        for (int x = 0; x < bw; ++x) printf(x ? " %d" : "%d", gob[y * bw + x]);
        printf("\n");
    }
    free(lost);
    free(gob);
    free(gptr);
    free(ids);
    return 0;
}
