"""CPU oracle of the grid-filtered spatial join (test infrastructure only)."""
