/* A C11 client of include/fipt.h that needs no GPU: it checks that the
 * header stands alone as C, that the library links, and that the
 * host-side entry points answer as the header documents. */
#include <stddef.h>
#include <stdio.h>
#include <string.h>

#include "fipt.h"

#define CHECK(c)                                                        \
    do {                                                                \
        if (!(c)) {                                                     \
            fprintf(stderr, "check failed at line %d: %s\n", __LINE__, #c); \
            return 1;                                                   \
        }                                                               \
    } while (0)

int main(void)
{
    /* the 40-byte query record the bake reads */
    CHECK(sizeof(fipt_query) == 40);
    CHECK(offsetof(fipt_query, n) == 12 && offsetof(fipt_query, wo) == 24);
    CHECK(offsetof(fipt_query, tri) == 36);

    CHECK(strncmp(fipt_version(), "fipt-gb300", 10) == 0);
    CHECK(strcmp(fipt_status_string(FIPT_OK), "ok") == 0);
    CHECK(strcmp(fipt_status_string(FIPT_ERR_WORKSPACE), "workspace too small") == 0);

    /* workspace queries are pure host arithmetic */
    size_t bytes = 0;
    CHECK(fipt_scene_workspace_size(100, 36, &bytes) == FIPT_OK && bytes > 36 * 144);
    CHECK(fipt_scene_workspace_size(-1, 36, &bytes) == FIPT_ERR_INVALID_ARG);
    CHECK(strlen(fipt_last_error()) > 0);
    CHECK(fipt_tri_error_workspace_size(1000, 10, &bytes) == FIPT_OK && bytes > 0);
    CHECK(fipt_voxel_cache_workspace_size(1000, &bytes) == FIPT_OK && bytes > 0);
    CHECK(fipt_emitter_radiance_workspace_size(1000, 10, &bytes) == FIPT_OK && bytes > 0);
    fipt_bake_params bp;
    memset(&bp, 0, sizeof(bp));
    bp.K = 6;
    bp.spp_diffuse = 32;
    bp.spp_specular = 32;
    CHECK(fipt_bake_refine_workspace_size(1000, &bp, 8, &bytes) == FIPT_OK && bytes >= 1000u * 224u * 184u);
    bp.spp_diffuse = 1 << 24;
    CHECK(fipt_bake_refine_workspace_size(1, &bp, 8, &bytes) == FIPT_ERR_INVALID_ARG);
    CHECK(fipt_render_grad_scale(0, NULL, NULL, NULL, NULL, NULL) == FIPT_OK);

    /* NULL arguments are rejected before any device work */
    CHECK(fipt_bake(NULL, NULL, 0, NULL, NULL, NULL, NULL, NULL) == FIPT_ERR_INVALID_ARG);
    CHECK(fipt_emitter_classify(NULL, 5, 100, 0.01f, NULL, NULL, NULL) == FIPT_ERR_INVALID_ARG);

    /* the admission arena: first fit, coalescing, budget errors */
    fipt_arena* a = NULL;
    CHECK(fipt_arena_create(4096, &a) == FIPT_OK && a);
    size_t o1, o2, o3, used, peak, largest;
    CHECK(fipt_arena_alloc(a, 1000, &o1) == FIPT_OK);
    CHECK(fipt_arena_alloc(a, 1000, &o2) == FIPT_OK && o2 != o1);
    CHECK(fipt_arena_alloc(a, 4096, &o3) == FIPT_ERR_BUDGET);
    CHECK(fipt_arena_free(a, o1, 1000) == FIPT_OK);
    CHECK(fipt_arena_free(a, o2, 1000) == FIPT_OK);
    CHECK(fipt_arena_info(a, &used, &peak, &largest) == FIPT_OK);
    CHECK(used == 0 && peak >= 2000 && largest == 4096);
    CHECK(fipt_arena_destroy(a) == FIPT_OK);

    puts("abi host checks ok");
    return 0;
}
