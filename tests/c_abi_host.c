/* A plain C caller of libcdr: the header compiles as C99 and the library links
 * without C++ or PyTorch. Only calls that need no GPU are made: status texts,
 * the device architecture tag, and argument checks that fail on the host.
 * Prints one line per check and returns 0 when every check holds. */
#include <stdio.h>
#include <string.h>

#include "cdr.h"

static int fails = 0;

static void expect(int got, int want, const char* what) {
  printf("%s: %d (%s)\n", what, got, cdr_status_string(got));
  if (got != want) ++fails;
}

static void check(int cond, const char* what) {
  printf("%s: %s\n", what, cond ? "yes" : "no");
  if (!cond) ++fails;
}

int main(void) {
  cdr_handle* h = NULL;
  /* the unit cube's 8 corners as one tetrahedron with an out-of-range index */
  double xyz[8 * 3] = {0};
  int32_t tets[4] = {0, 1, 2, 8};
  cdr_mesh_in in;
  memset(&in, 0, sizeof in);
  in.xyz = xyz;
  in.n_verts = 8;
  in.tets = tets;
  in.n_tets = 1;
  check(cdr_device_arch() == 103, "built for sm_103a");
  expect(cdr_create(NULL, NULL, NULL, NULL, &h), CDR_ERR_INVALID_INPUT, "create without input");
  expect(cdr_create(&in, NULL, NULL, NULL, &h), CDR_ERR_INVALID_INPUT, "create, bad index");
  check(h == NULL, "no handle made");
  expect(cdr_refine(NULL, 2.0, 1, NULL), CDR_ERR_INVALID_INPUT, "refine without handle");
  expect(cdr_delaunay_box(xyz, 7, NULL, NULL, NULL, &h, NULL, NULL), CDR_ERR_INVALID_INPUT,
         "delaunay with 7 points");
  cdr_destroy(NULL);
  printf("%s\n", fails ? "FAILED" : "ok");
  return fails ? 1 : 0;
}
