/* A plain C client of the library's C ABI (include/cse.h), used by
 * tests/test_c_client.py to show that the boundary needs nothing but C.
 *
 *   c_client checks           argument checks that need no device, and the
 *                             status of a device call (prints "device <code>")
 *   c_client search FILE      loads the matrices in FILE, runs one search and
 *                             prints the total and each matrix's Cost and list
 *   c_client sizes            prints the size and the offset of the last field
 *                             of every struct the header declares
 *
 * FILE (little-endian int32 header, then int8 entries):
 *   n_mats, n_proc, seed_lo, seed_hi, budget, interval, permille, cap,
 *   7 strategy weights, then per matrix rows, cols and rows * cols entries. */
#include <stddef.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "cse.h"

static int expect(const char* what, int got, int want) {
    if (got != want) {
        printf("FAIL %s: %d, expected %d (%s)\n", what, got, want, cse_last_error());
        return 1;
    }
    return 0;
}

static int checks(void) {
    int bad = 0;
    cse_opts o;
    cse_opts_default(&o);
    bad |= expect("default interval", (int)o.share_interval, 32);
    bad |= expect("default permille", (int)o.share_permille, 400);
    bad |= expect("default cap", (int)o.col_cap, 128);

    const int8_t bad_entry[4] = {1, 2, 0, 1};
    const int8_t* mats[1] = {bad_entry};
    const int32_t rows[1] = {2}, cols[1] = {2};
    cse_scheme* s = NULL;
    bad |= expect("non-ternary entry", cse_scheme_load(mats, rows, cols, 1, &s), CSE_EINVAL);
    bad |= expect("no output", cse_scheme_load(mats, rows, cols, 1, NULL), CSE_EINVAL);
    bad |= expect("philox n < 0", cse_philox(0, NULL, -1, NULL), CSE_EINVAL);
    bad |= expect("philox n = 0", cse_philox(0, NULL, 0, NULL), CSE_OK);

    const int8_t ok[6] = {1, 1, 0, 1, -1, 1};
    const int8_t* mats2[1] = {ok};
    const int32_t rows2[1] = {2}, cols2[1] = {3};
    int rc = cse_scheme_load(mats2, rows2, cols2, 1, &s);
    printf("device %d\n", rc);
    if (rc == CSE_OK) cse_scheme_free(s);
    printf(bad ? "checks failed\n" : "checks ok\n");
    return bad;
}

static int search(const char* path) {
    FILE* f = fopen(path, "rb");
    if (!f) {
        printf("cannot open %s\n", path);
        return 1;
    }
    int32_t h[15];
    if (fread(h, 4, 15, f) != 15) {
        fclose(f);
        return 1;
    }
    const int n = h[0];
    if (n < 1 || n > CSE_MAX_MATS) {
        fclose(f);
        return 1;
    }
    int8_t* data[CSE_MAX_MATS];
    const int8_t* mats[CSE_MAX_MATS];
    int32_t rows[CSE_MAX_MATS], cols[CSE_MAX_MATS];
    for (int k = 0; k < n; k++) {
        int32_t rc2[2];
        if (fread(rc2, 4, 2, f) != 2) {
            fclose(f);
            return 1;
        }
        rows[k] = rc2[0];
        cols[k] = rc2[1];
        data[k] = (int8_t*)malloc((size_t)rows[k] * (size_t)cols[k]);
        if (!data[k] || fread(data[k], 1, (size_t)rows[k] * (size_t)cols[k], f) != (size_t)rows[k] * (size_t)cols[k]) {
            fclose(f);
            return 1;
        }
        mats[k] = data[k];
    }
    fclose(f);
    cse_strategy_mix mix = {(uint32_t)h[8], (uint32_t)h[9], (uint32_t)h[10], (uint32_t)h[11],
                            (uint32_t)h[12], (uint32_t)h[13], (uint32_t)h[14]};
    cse_opts o;
    cse_opts_default(&o);
    o.share_interval = (uint32_t)h[5];
    o.share_permille = (uint32_t)h[6];
    o.col_cap = (uint32_t)h[7];
    const uint64_t seed = (uint64_t)(uint32_t)h[2] | (uint64_t)(uint32_t)h[3] << 32;

    cse_scheme* s = NULL;
    cse_result* r = NULL;
    int rc = cse_scheme_load(mats, rows, cols, n, &s);
    if (rc == CSE_OK) rc = cse_search(s, &mix, h[1], seed, h[4], &o, NULL, &r);
    int32_t* list = (int32_t*)malloc((size_t)o.col_cap * sizeof(int32_t));
    for (int k = 0; rc == CSE_OK && k < n; k++) {
        int32_t len = 0;
        int64_t add = 0, total = 0;
        rc = cse_result_fetch(r, k, list, (int32_t)o.col_cap, &len, &add, &total);
        if (rc != CSE_OK) break;
        if (k == 0) printf("total %lld\n", (long long)total);
        printf("matrix %d cost %lld list", k, (long long)add);
        for (int e = 0; e < len; e++) printf(" %d", list[e]);
        printf("\n");
    }
    if (rc != CSE_OK) printf("error %d: %s\n", rc, cse_last_error());
    free(list);
    cse_result_free(r);
    cse_scheme_free(s);
    for (int k = 0; k < n; k++) free(data[k]);
    return rc != CSE_OK;
}

static int sizes(void) {
    printf("cse_strategy_mix %zu %zu\n", sizeof(cse_strategy_mix), offsetof(cse_strategy_mix, w_gp));
    printf("cse_opts %zu %zu\n", sizeof(cse_opts), offsetof(cse_opts, cta_min_list));
    printf("cse_tune_entry %zu %zu\n", sizeof(cse_tune_entry), offsetof(cse_tune_entry, trial_ms_wide));
    printf("cse_proc_record %zu %zu\n", sizeof(cse_proc_record), offsetof(cse_proc_record, method_ops));
    return 0;
}

int main(int argc, char** argv) {
    if (argc >= 2 && strcmp(argv[1], "checks") == 0) return checks();
    if (argc >= 2 && strcmp(argv[1], "sizes") == 0) return sizes();
    if (argc >= 3 && strcmp(argv[1], "search") == 0) return search(argv[2]);
    printf("usage: %s checks | search FILE | sizes\n", argv[0]);
    return 2;
}
