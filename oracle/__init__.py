"""CPU oracle (test infrastructure only): plain FP64 restatement of the method, no CUDA."""
