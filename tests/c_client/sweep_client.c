/*
 * A plain C11 client of the SU(Nc) link-sweep library: it uses nothing but the
 * public header and libsun.so (no Python, no PyTorch), to show that the C ABI
 * stands on its own.
 *
 *   sweep_client NC NX NY NZ NT BETA SEED SWEEPS N_HB N_OR OUT
 *
 * creates a hot-start lattice with library-owned device memory and stream,
 * runs SWEEPS sweeps of N_HB heatbath and N_OR overrelaxation steps (Sec. 3)
 * with the plaquette (Eq. 4) and Polyakov loop measured after each, checks the
 * links' health, and writes OUT as raw little-endian doubles:
 *   plaquette history [SWEEPS], Polyakov history [2*SWEEPS] (re, im),
 *   links in canonical order [8*NC*NC*V].
 * It also checks that a call with invalid arguments fails with a status and a
 * message, without aborting.  Exit 0 on success, 1 on any failure.
 */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "sun.h"

#define CHECK(call)                                                                  \
  do {                                                                               \
    sun_status st_ = (call);                                                         \
    if (st_ != SUN_OK) {                                                             \
      fprintf(stderr, "%s failed: %s (%s)\n", #call, sun_status_string(st_),         \
              sun_last_error());                                                     \
      goto fail;                                                                     \
    }                                                                                \
  } while (0)

int main(int argc, char** argv) {
  sun_lattice* lat = NULL;
  double *plaq = NULL, *poly = NULL, *links = NULL;
  FILE* out = NULL;
  int rc = 1;
  if (argc != 12) {
    fprintf(stderr, "usage: %s NC NX NY NZ NT BETA SEED SWEEPS N_HB N_OR OUT\n", argv[0]);
    return 1;
  }
  const int nc = atoi(argv[1]);
  const int dims[4] = {atoi(argv[2]), atoi(argv[3]), atoi(argv[4]), atoi(argv[5])};
  const double beta = atof(argv[6]);
  const uint64_t seed = strtoull(argv[7], NULL, 10);
  const int sweeps = atoi(argv[8]), n_hb = atoi(argv[9]), n_or = atoi(argv[10]);
  const size_t volume = (size_t)dims[0] * dims[1] * dims[2] * dims[3];
  const size_t n_links = 8u * (size_t)nc * nc * volume;

  if (sun_abi_version() != SUN_ABI_VERSION) {
    fprintf(stderr, "ABI version %d, header %d\n", sun_abi_version(), SUN_ABI_VERSION);
    return 1;
  }

  /* invalid arguments come back as a status and a message */
  {
    const int odd[4] = {3, 4, 4, 4};
    sun_lattice* bad = NULL;
    sun_status st = sun_lattice_create(&bad, 3, odd, 6.0, 0, 1, NULL);
    if (st != SUN_ERR_ARG || bad != NULL || sun_last_error()[0] == '\0') {
      fprintf(stderr, "an odd extent was not rejected cleanly (status %d)\n", (int)st);
      return 1;
    }
  }

  sun_options opt;
  sun_options_init(&opt);
  if (sun_footprint_bytes(nc, dims, &opt) == 0) {
    fprintf(stderr, "no footprint for these arguments\n");
    return 1;
  }
  CHECK(sun_lattice_create(&lat, nc, dims, beta, 1, seed, &opt));

  plaq = (double*)malloc(sizeof(double) * (size_t)sweeps);
  poly = (double*)malloc(sizeof(double) * 2u * (size_t)sweeps);
  /* export wants a 16-byte aligned host buffer */
  links = (double*)aligned_alloc(64, ((sizeof(double) * n_links + 63) / 64) * 64);
  if (!plaq || !poly || !links) {
    fprintf(stderr, "out of host memory\n");
    goto fail;
  }
  CHECK(sun_run(lat, sweeps, n_hb, n_or, plaq, poly));

  {
    double dev_u = 0, dev_det = 0;
    uint64_t n_bad = 0;
    CHECK(sun_check_links(lat, &dev_u, &dev_det, &n_bad));
    if (n_bad != 0 || dev_u > 1e-4 || dev_det > 1e-4) {
      fprintf(stderr, "unhealthy links: %g %g %llu\n", dev_u, dev_det, (unsigned long long)n_bad);
      goto fail;
    }
  }
  CHECK(sun_export_links(lat, links, n_links));

  out = fopen(argv[11], "wb");
  if (!out) {
    fprintf(stderr, "cannot open %s\n", argv[11]);
    goto fail;
  }
  if (fwrite(plaq, sizeof(double), (size_t)sweeps, out) != (size_t)sweeps ||
      fwrite(poly, sizeof(double), 2u * (size_t)sweeps, out) != 2u * (size_t)sweeps ||
      fwrite(links, sizeof(double), n_links, out) != n_links) {
    fprintf(stderr, "short write to %s\n", argv[11]);
    goto fail;
  }
  printf("plaquette %.17g\n", plaq[sweeps - 1]);
  rc = 0;

fail:
  if (out && fclose(out) != 0) rc = 1;
  sun_lattice_destroy(lat);
  free(plaq);
  free(poly);
  free(links);
  return rc;
}
