#!/bin/bash
# Build and run the MUFU/FFMA/DFMA throughput probe (needs a GPU).
set -e
HERE="$(cd "$(dirname "$0")" && pwd)"
/usr/local/cuda/bin/nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o "$HERE/probe_rates" "$HERE/probe_rates.cu"
"$HERE/probe_rates"
