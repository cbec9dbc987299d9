/* The C ABI from plain C, without Python or a GPU: pattern validation,
 * host-only plans (graph NULL), the matched (alternative) set and the morph
 * transform, checked on a data graph whose counts have a closed form.
 *
 * On the complete graph K_k every connected k-vertex pattern p occurs
 * k!/|Aut(p)| times edge-induced, while vertex-induced only the clique
 * occurs, once.  Feeding the matched patterns' counts on K_k into pm_morph
 * must give those values for every vertex- and edge-induced query
 * (Theorem 3.1 and Corollary 3.1 applied to a graph where both sides are
 * known).
 *
 * Build: gcc -std=c11 -I include tests/c_abi_check.c -L<lib dir> -lpm_b300
 * Prints "ok" and exits 0 when every check holds. */
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "pm.h"

static int failures = 0;

#define CHECK(cond, ...)                      \
    do {                                      \
        if (!(cond)) {                        \
            fprintf(stderr, __VA_ARGS__);     \
            fputc('\n', stderr);              \
            failures++;                       \
        }                                     \
    } while (0)

/* bit of pair (a, b), a < b, in the lexicographic pair order */
static int pair_bit(int k, int a, int b) {
    if (a > b) { int t = a; a = b; b = t; }
    return a * (2 * k - a - 1) / 2 + (b - a - 1);
}

static int has_edge(uint32_t mask, int k, int a, int b) { return (mask >> pair_bit(k, a, b)) & 1u; }

static int connected(int k, uint32_t mask) {
    int seen = 1, grew = 1;
    while (grew) {
        grew = 0;
        for (int v = 0; v < k; v++)
            if (seen >> v & 1)
                for (int u = 0; u < k; u++)
                    if (!(seen >> u & 1) && has_edge(mask, k, u, v)) { seen |= 1 << u; grew = 1; }
    }
    return seen == (1 << k) - 1;
}

/* |Aut| by trying every permutation (k <= 6: at most 720) */
static int count_aut(int k, uint32_t mask, int *perm, int depth, int used) {
    if (depth == k) {
        for (int a = 0; a < k; a++)
            for (int b = a + 1; b < k; b++)
                if (has_edge(mask, k, a, b) != has_edge(mask, k, perm[a], perm[b])) return 0;
        return 1;
    }
    int total = 0;
    for (int x = 0; x < k; x++) {
        if (used >> x & 1) continue;
        perm[depth] = x;
        total += count_aut(k, mask, perm, depth + 1, used | (1 << x));
    }
    return total;
}

static uint64_t count_on_clique(int k, uint32_t mask, int induced) {
    const uint32_t full = (1u << (k * (k - 1) / 2)) - 1;
    if (induced == PM_VERTEX_INDUCED && mask != full) return 0;
    int perm[PM_MAX_K];
    uint64_t fact = 1;
    for (int i = 2; i <= k; i++) fact *= (uint64_t)i;
    return fact / (uint64_t)count_aut(k, mask, perm, 0, 0);
}

static pm_pattern make(int k, uint32_t mask, int induced) {
    pm_pattern p;
    memset(&p, 0, sizeof p);
    p.k = k;
    p.edge_mask = mask;
    p.induced = induced;
    for (int i = 0; i < PM_MAX_K; i++) p.label[i] = -1;
    return p;
}

static void check_morph_on_clique(int k, int induced) {
    static pm_pattern q[1 << 15], matched[1 << 12];
    static uint64_t mcount[2 << 12], req[2 << 15];
    int nq = 0;
    for (uint32_t m = 0; m < (1u << (k * (k - 1) / 2)); m++)
        if (connected(k, m)) q[nq++] = make(k, m, induced);
    pm_query_plan *p = NULL;
    pm_status st = pm_plan(NULL, q, nq, PM_OP_COUNT, PM_MORPH_NAIVE, &p);
    CHECK(st == PM_OK, "pm_plan(k=%d): %s", k, pm_strerror(st));
    if (st != PM_OK) return;
    pm_plan_info info;
    CHECK(pm_plan_get_info(p, &info) == PM_OK && info.n_queries == nq, "pm_plan_get_info");
    CHECK(info.n_matched > 0 && info.n_matched <= (1 << 12), "n_matched %d", info.n_matched);
    CHECK(pm_plan_matched(p, matched) == PM_OK, "pm_plan_matched");
    for (int j = 0; j < info.n_matched; j++) {
        mcount[2 * j] = count_on_clique(matched[j].k, matched[j].edge_mask, matched[j].induced);
        mcount[2 * j + 1] = 0;
    }
    CHECK(pm_morph(p, mcount, req) == PM_OK, "pm_morph");
    for (int i = 0; i < nq; i++) {
        const uint64_t want = count_on_clique(k, q[i].edge_mask, induced);
        CHECK(req[2 * i] == want && req[2 * i + 1] == 0,
              "k=%d %s query mask %u: morphed %llu, closed form %llu", k,
              induced == PM_VERTEX_INDUCED ? "vertex-induced" : "edge-induced", q[i].edge_mask,
              (unsigned long long)req[2 * i], (unsigned long long)want);
    }
    /* a plan without a graph cannot run */
    CHECK(pm_count(p, NULL, 0.0, req, NULL) == PM_EINVAL,
          "pm_count without a graph must fail with PM_EINVAL");
    pm_free_plan(p);
}

int main(void) {
    /* pattern validation: statuses, never aborts */
    pm_query_plan *p = NULL;
    pm_pattern bad = make(4, (1u << pair_bit(4, 0, 1)) | (1u << pair_bit(4, 2, 3)), PM_EDGE_INDUCED);
    CHECK(pm_plan(NULL, &bad, 1, PM_OP_COUNT, PM_MORPH_NONE, &p) == PM_EINVAL,
          "a disconnected pattern must be rejected");
    pm_pattern big = make(9, 1, PM_EDGE_INDUCED);
    CHECK(pm_plan(NULL, &big, 1, PM_OP_COUNT, PM_MORPH_NONE, &p) == PM_EINVAL,
          "k = 9 must be rejected");
    CHECK(pm_strerror(PM_ETIMEOUT) != NULL && strlen(pm_strerror(PM_ETIMEOUT)) > 0, "pm_strerror");
    for (int k = 3; k <= 6; k++) {
        check_morph_on_clique(k, PM_VERTEX_INDUCED);
        check_morph_on_clique(k, PM_EDGE_INDUCED);
    }
    if (failures) {
        fprintf(stderr, "%d check(s) failed\n", failures);
        return 1;
    }
    printf("ok\n");
    return 0;
}
