"""FP64 CPU oracle of the Mu3e online event selection: test infrastructure only."""
