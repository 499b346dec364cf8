/* Prints sizeof / offsetof of the public ABI structs, for the binding test. */
#include <stddef.h>
#include <stdio.h>
#include "colt.h"
int main(void) {
  printf("colt_grid_desc %zu\n", sizeof(colt_grid_desc));
  printf("colt_camera %zu\n", sizeof(colt_camera));
  printf("colt_run_params %zu\n", sizeof(colt_run_params));
  printf("colt_result %zu\n", sizeof(colt_result));
  printf("colt_stats %zu\n", sizeof(colt_stats));
  printf("colt_launch_config %zu\n", sizeof(colt_launch_config));
  printf("colt_scatter_io %zu\n", sizeof(colt_scatter_io));
  printf("off_scatter_n_trials %zu\n", offsetof(colt_scatter_io, n_trials));
  printf("off_run_precision %zu\n", offsetof(colt_run_params, precision));
  printf("off_run_emission %zu\n", offsetof(colt_run_params, emission));
  printf("off_run_source %zu\n", offsetof(colt_run_params, source));
  printf("off_result_pk_freq %zu\n", offsetof(colt_result, pk_freq));
  printf("colt_source %zu\n", sizeof(colt_source));
  printf("off_run_sources %zu\n", offsetof(colt_run_params, sources));
  printf("off_stats_kernel_ms %zu\n", offsetof(colt_stats, ctx_kernel_ms));
  printf("off_stats_longest %zu\n", offsetof(colt_stats, longest_history));
  printf("off_stats_peel_visits %zu\n", offsetof(colt_stats, ctx_peel_visits));
  printf("off_launch_refill_min %zu\n", offsetof(colt_launch_config, refill_min));
  return 0;
}
