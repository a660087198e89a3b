/* oracle_driver.c -- runs the C oracle (parse, tableau reference, per-shot
 * frame sampling of a few shots) over a corpus of circuits, for
 * address/undefined-behaviour sanitizer builds (tests/test_sanitizers.py).
 * Circuits are separated by lines "%%". Exits non-zero only on a sanitizer
 * report (the sanitizers abort). */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef struct orc_circuit orc_circuit;
int orc_parse(const char *text, orc_circuit **out, char *err, size_t errlen);
void orc_info(const orc_circuit *c, uint64_t out[7]);
int orc_reference(const orc_circuit *c, uint8_t *ref, uint8_t *detflag);
int orc_frame_shots(const orc_circuit *c, const uint8_t *ref, uint64_t seed, uint64_t shot_offset,
                    const uint64_t *shots, size_t nshots, uint8_t *meas, uint8_t *dets, int nthreads);
void orc_free(orc_circuit *c);

int main(int argc, char **argv) {
    if (argc < 2) return 2;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 2;
    fseek(f, 0, SEEK_END);
    long len = ftell(f);
    fseek(f, 0, SEEK_SET);
    char *all = (char *)malloc((size_t)len + 1);
    if (fread(all, 1, (size_t)len, f) != (size_t)len) return 2;
    all[len] = 0;
    fclose(f);
    int ok = 0, rejected = 0;
    char *p = all;
    for (;;) {
        char *sep = strstr(p, "\n%%\n");
        if (sep) *sep = 0;
        orc_circuit *c = NULL;
        char err[256];
        if (orc_parse(p, &c, err, sizeof err) != 0) {
            rejected++;
        } else {
            uint64_t info[7];
            orc_info(c, info);
            const uint64_t M = info[1], D = info[2] + info[6];
            uint8_t *ref = (uint8_t *)calloc(M + 1, 1), *det = (uint8_t *)calloc(M + 1, 1);
            uint64_t shots[5] = {0, 1, 63, 64, 200};
            uint8_t *meas = (uint8_t *)calloc(5 * (M + 1), 1), *dets = (uint8_t *)calloc(5 * (D + 1), 1);
            if (orc_reference(c, ref, det) == 0) orc_frame_shots(c, ref, 7, 64, shots, 5, meas, dets, 2);
            free(ref);
            free(det);
            free(meas);
            free(dets);
            orc_free(c);
            ok++;
        }
        if (!sep) break;
        p = sep + 4;
    }
    free(all);
    printf("sampled %d rejected %d\n", ok, rejected);
    return 0;
}
