// Host reader/packer for RDEMECH 1 text (see mech_layout.h for the image).
#pragma once
#include <stddef.h>

#include <string>
#include <vector>

#include "mech_layout.h"

namespace rde {

// Returns 0 on success, -1 on a syntax error, -2 on an inconsistent mechanism;
// *err receives a one-line description on failure.
// E_J, if given, receives each reaction's activation energy in J/mol (of k_inf for falloff).
int pack_mechanism(const char* text, size_t len, std::vector<unsigned char>* image, std::string* err,
                   std::vector<double>* E_J = nullptr);

// Gather plan of the CTA-per-cell kernel (large_plan.h) for a packed image.
void build_large_plan(const unsigned char* image, std::vector<unsigned char>* plan);

}  // namespace rde
