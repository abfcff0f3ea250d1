/* The C usage example of the library: estimate a disparity map from two host
 * RGB images with the paper's settings (10 outer iterations).  Compiled and
 * linked against include/lem.h and the in-tree liblem.so by tests/test_abi.py;
 * running it needs a GPU. */
#include <stdint.h>
#include <stdio.h>

#include "lem.h"

int example(const uint8_t *left_rgb, const uint8_t *right_rgb, int H, int W, float *disparity_host);

int example(const uint8_t *left_rgb, const uint8_t *right_rgb, int H, int W, float *disparity_host) {
    lem_params p;
    lem_default_params(&p);
    p.disp_max = 60.0;
    /* host images, packed 8-bit RGB */
    lem_image L = {left_rgb, H, W, 3 * W, 0, 3, 3, LEM_IMG_U8}, R = {right_rgb, H, W, 3 * W, 0, 3, 3, LEM_IMG_U8};
    lem_handle *h = NULL;
    if (lem_create(&L, &R, &p, &h) != LEM_OK) {
        fprintf(stderr, "%s\n", lem_last_error(NULL));
        return 1;
    }
    lem_stats st;
    lem_expand_iteration(h, 10, &st);                 /* st.energy, st.evals, ... */
    lem_get_labels(h, NULL, disparity_host, NULL, 0); /* H*W floats on the host */
    lem_destroy(h);
    return 0;
}

int main(void) { return 0; }
